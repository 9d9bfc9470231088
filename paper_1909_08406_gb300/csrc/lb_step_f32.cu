// FP32-arithmetic step kernels (FP32, FP16 and BF16 storage).  Variants:
//   kKernelDirect1   k_step:        one node per thread, direct global loads
//   kKernelDirect2   k_step2<.,.,3>: two rows per thread, packed FP32x2 math
//   kKernelDirect2R  k_step2<.,.,4>: the same, register budget for 4 CTAs/SM
//   kKernelStaged    k_step_tma:    rows fetched by TMA bulk copies into a
//                                   shared-memory ring
//   kKernelWarpSpec  k_step_ws:     the same staging with a dedicated producer
//                                   warp, full/empty mbarriers, and consumers
//                                   updating two rows per thread (FP32x2)
// This unit is compiled with ptxas double-precision-use warnings so that no
// FP64 instruction slips into the float path.
#include "lb_kernels.cuh"
#include "lb_step_tma.cuh"
#include "lb_step_ws.cuh"

namespace gblb {

template <class Codec, bool P>
static cudaError_t run_direct1(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta,
                               int* err, cudaStream_t st) {
    using T = typename Codec::raw_t;
    const int th = step_threads(d);
    k_step<Codec, P><<<step_grid(d, th), th, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                      (float)twobeta, err);
    return cudaGetLastError();
}

template <class Codec, bool P, int MINB>
static cudaError_t run_direct2(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta,
                               int* err, cudaStream_t st) {
    using T = typename Codec::raw_t;
    const int th = step_threads(d);
    const int chunks = (d.nx + th - 1) / th;
    const int64_t blocks = d.rows / 2 * chunks;
    k_step2<Codec, P, MINB><<<(unsigned)blocks, th, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d,
                                                             c.kf, (float)twobeta, err, chunks);
    return cudaGetLastError();
}

template <class Codec, bool P, int MINB, int MODE, bool SR = false>
static cudaError_t run_direct2x(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta,
                                int* err, cudaStream_t st, int rpb, uint32_t sr_key = 0) {
    using T = typename Codec::raw_t;
    if constexpr (sizeof(T) != 2) {
        return cudaErrorInvalidValue;
    } else {
        const int half = d.nx / 2;
        const int th = half >= 128 ? 128 : ((half + 31) / 32) * 32;
        const int chunks = (half + th - 1) / th;
        const int64_t blocks = ((d.rows + rpb - 1) / rpb) * chunks;
        auto kern = k_step2x<Codec, P, MINB, MODE, SR>;
        kern<<<(unsigned)blocks, th, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                 (float)twobeta, err, chunks, rpb, sr_key);
        return cudaGetLastError();
    }
}

// Per-instance launch data: dynamic shared memory opt-in and the persistent grid size.
struct TmaLaunchInfo {
    int device = -1;
    int grid = 0;
};

template <class Codec, bool P, class Cfg>
static cudaError_t run_tma(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta, int* err,
                           cudaStream_t st) {
    using T = typename Codec::raw_t;
    static TmaLaunchInfo info;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto kern = k_step_tma<Codec, P, Cfg>;
    if (info.device != dev) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::THREADS, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        info.grid = per_sm * sms;
        info.device = dev;
    }
    const int64_t ntiles = d.rows * (d.nx / Cfg::TX);
    const int grid = (int)(ntiles < info.grid ? ntiles : info.grid);
    const long long wait_limit = 4000000000LL;  // ~2 s of SM clock
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                 (float)twobeta, err, wait_limit);
    return cudaGetLastError();
}

template <class Codec, bool P, class Cfg>
static cudaError_t run_ws(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta, int* err,
                          cudaStream_t st) {
    using T = typename Codec::raw_t;
    static TmaLaunchInfo info;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto kern = k_step_ws<Codec, P, Cfg>;
    if (info.device != dev) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::THREADS, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        info.grid = per_sm * sms;
        info.device = dev;
    }
    const int64_t ntiles = d.rows / 2 * (d.nx / Cfg::TX);
    const int grid = (int)(ntiles < info.grid ? ntiles : info.grid);
    const long long wait_limit = 4000000000LL;  // ~2 s of SM clock
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                 (float)twobeta, err, wait_limit);
    return cudaGetLastError();
}

// Warp-specialised shapes: 128 x per tile, 4 consumer warps.  16-bit: 70.8 KB ring
// (3 stages) -> up to 3 CTAs/SM; FP32: 89.3 KB ring (2 stages) -> 2 CTAs/SM.
template <class Codec>
struct WsShape {
    using Cfg = WsCfg<Codec, 128, 4, (sizeof(typename Codec::raw_t) == 2 ? 3 : 2),
                      (sizeof(typename Codec::raw_t) == 2 ? 3 : 2)>;
};

// Staged-kernel shapes per storage type: (tile width, threads, ring depth, CTAs/SM).
// FP32, TX 256: 86.6 KB ring -> 2 CTAs/SM; TX 128: 66.9 KB -> 3 CTAs/SM.
// 16-bit, TX 256: 66.9 KB -> 3 CTAs/SM; TX 128: 47.3 KB -> 4 CTAs/SM.
template <class Codec, int TX>
struct TmaShape;
template <int TX>
struct TmaShape<CodecF32, TX> {
    using Cfg = TmaCfg<CodecF32, TX, (TX < 256 ? TX : 256), (TX >= 256 ? 2 : 3), (TX >= 256 ? 2 : 3)>;
};
template <int TX>
struct TmaShape<CodecF16, TX> {
    using Cfg = TmaCfg<CodecF16, TX, (TX < 256 ? TX : 256), (TX >= 256 ? 3 : 4), (TX >= 256 ? 3 : 4)>;
};
template <int TX>
struct TmaShape<CodecBF16, TX> {
    using Cfg = TmaCfg<CodecBF16, TX, (TX < 256 ? TX : 256), (TX >= 256 ? 3 : 4), (TX >= 256 ? 3 : 4)>;
};

int tma_tile_width(int prec, const Dims& d) {
    if (prec == kF64) return 0;
    const size_t es = storage_bytes(prec);
    if (((size_t)d.nx * es) % 16 != 0) return 0;
    if (d.nx % 256 == 0) return 256;
    if (d.nx % 128 == 0) return 128;
    return 0;
}

int resolve_kernel(int prec, const Dims& d, int kernel) {
    if (prec == kF64) return kKernelDirect1;
    const bool two_rows = d.ny % 2 == 0 && d.plane < ((int64_t)1 << 32);
    switch (kernel) {
        case kKernelDirect2X:
        case kKernelDirect2XL:
            return (storage_bytes(prec) == 2 && d.nx % 2 == 0 && d.plane < ((int64_t)1 << 32))
                       ? kernel
                       : resolve_kernel(prec, d, kKernelAuto);
        case kKernelWarpSpec:
            return (two_rows && d.nx % 128 == 0 && tma_tile_width(prec, d)) ? kKernelWarpSpec
                                                                             : resolve_kernel(prec, d, kKernelAuto);
        case kKernelStaged: return tma_tile_width(prec, d) ? kKernelStaged : resolve_kernel(prec, d, kKernelAuto);
        case kKernelDirect2:
        case kKernelDirect2R: return two_rows ? kernel : kKernelDirect1;
        case kKernelDirect1: return kKernelDirect1;
        default:
            if (storage_bytes(prec) == 2 && d.nx % 2 == 0 && d.plane < ((int64_t)1 << 32)) return kKernelDirect2XL;
            return two_rows ? kKernelDirect2 : kKernelDirect1;
    }
}

template <class Codec, bool P>
static cudaError_t step_codec(int prec, int kernel, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                              double twobeta, int* err, cudaStream_t st) {
    switch (resolve_kernel(prec, d, kernel)) {
        case kKernelStaged:
            if (tma_tile_width(prec, d) == 256)
                return run_tma<Codec, P, typename TmaShape<Codec, 256>::Cfg>(src, dst, d, c, twobeta, err, st);
            return run_tma<Codec, P, typename TmaShape<Codec, 128>::Cfg>(src, dst, d, c, twobeta, err, st);
        case kKernelWarpSpec: return run_ws<Codec, P, typename WsShape<Codec>::Cfg>(src, dst, d, c, twobeta, err, st);
        case kKernelDirect2X: return run_direct2x<Codec, P, 3, 0>(src, dst, d, c, twobeta, err, st, 1);
        case kKernelDirect2XL: return run_direct2x<Codec, P, 3, 2>(src, dst, d, c, twobeta, err, st, 2);

        case kKernelDirect2: return run_direct2<Codec, P, 3>(src, dst, d, c, twobeta, err, st);
        case kKernelDirect2R: return run_direct2<Codec, P, 4>(src, dst, d, c, twobeta, err, st);
        default: return run_direct1<Codec, P>(src, dst, d, c, twobeta, err, st);
    }
}

cudaError_t launch_step_f32(int prec, bool project, int kernel, const void* src, void* dst, const Dims& d,
                            const LaunchConsts& c, double twobeta, int* err, cudaStream_t st) {
    switch (prec) {
        case kF32:
            return project ? step_codec<CodecF32, true>(prec, kernel, src, dst, d, c, twobeta, err, st)
                           : step_codec<CodecF32, false>(prec, kernel, src, dst, d, c, twobeta, err, st);
        case kF16:
            return project ? step_codec<CodecF16, true>(prec, kernel, src, dst, d, c, twobeta, err, st)
                           : step_codec<CodecF16, false>(prec, kernel, src, dst, d, c, twobeta, err, st);
        case kBF16:
            return project ? step_codec<CodecBF16, true>(prec, kernel, src, dst, d, c, twobeta, err, st)
                           : step_codec<CodecBF16, false>(prec, kernel, src, dst, d, c, twobeta, err, st);
        default: return cudaErrorInvalidValue;
    }
}

// The fused step with the stochastic BF16 store (series equilibrium with the momentum projection):
// the x-pair kernel where it applies, else one node per thread.
cudaError_t launch_step_sr(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta, int* err,
                           cudaStream_t st, uint32_t sr_key) {
    using T = CodecBF16::raw_t;
    if (resolve_kernel(kBF16, d, kKernelDirect2XL) == kKernelDirect2XL)
        return run_direct2x<CodecBF16, true, 3, 2, true>(src, dst, d, c, twobeta, err, st, 2, sr_key);
    const int th = step_threads(d);
    k_step_sr<CodecBF16><<<step_grid(d, th), th, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                         (float)twobeta, err, sr_key);
    return cudaGetLastError();
}

}  // namespace gblb
