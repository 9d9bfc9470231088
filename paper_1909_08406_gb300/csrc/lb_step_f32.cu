// FP32-arithmetic step kernels (FP32, FP16 and BF16 storage): the direct-load
// kernel and the shared-memory-staged (TMA bulk copy) kernel.  This unit is
// compiled with ptxas double-precision-use warnings so that no FP64
// instruction slips into the float path.
#include "lb_kernels.cuh"
#include "lb_step_tma.cuh"

namespace gblb {

template <class Codec, bool P>
static cudaError_t run(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta, int* err,
                       cudaStream_t st) {
    using T = typename Codec::raw_t;
    const int th = step_threads(d);
    k_step<Codec, P><<<step_grid(d, th), th, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                      (float)twobeta, err);
    return cudaGetLastError();
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

// Staged-kernel shapes per storage type: (tile width, threads, ring depth).
template <class Codec, int TX>
struct TmaShape;
// FP32, TX 256: 86.6 KB ring -> 2 CTAs/SM; TX 128: 66.9 KB -> 3 CTAs/SM.
// 16-bit, TX 256: 66.9 KB -> 3 CTAs/SM; TX 128: 47.3 KB -> 4 CTAs/SM.
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

template <class Codec, bool P>
static cudaError_t dispatch_tma(int tx, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                                double twobeta, int* err, cudaStream_t st) {
    if (tx == 256) return run_tma<Codec, P, typename TmaShape<Codec, 256>::Cfg>(src, dst, d, c, twobeta, err, st);
    if (tx == 128) return run_tma<Codec, P, typename TmaShape<Codec, 128>::Cfg>(src, dst, d, c, twobeta, err, st);
    return run<Codec, P>(src, dst, d, c, twobeta, err, st);
}

template <class Codec>
static cudaError_t step_codec(int prec, bool project, int variant, const void* src, void* dst, const Dims& d,
                              const LaunchConsts& c, double twobeta, int* err, cudaStream_t st) {
    const int tx = variant == kVariantStaged ? tma_tile_width(prec, d) : 0;
    if (tx)
        return project ? dispatch_tma<Codec, true>(tx, src, dst, d, c, twobeta, err, st)
                       : dispatch_tma<Codec, false>(tx, src, dst, d, c, twobeta, err, st);
    return project ? run<Codec, true>(src, dst, d, c, twobeta, err, st)
                   : run<Codec, false>(src, dst, d, c, twobeta, err, st);
}

cudaError_t launch_step_f32(int prec, bool project, int variant, const void* src, void* dst, const Dims& d,
                            const LaunchConsts& c, double twobeta, int* err, cudaStream_t st) {
    switch (prec) {
        case kF32: return step_codec<CodecF32>(prec, project, variant, src, dst, d, c, twobeta, err, st);
        case kF16: return step_codec<CodecF16>(prec, project, variant, src, dst, d, c, twobeta, err, st);
        case kBF16: return step_codec<CodecBF16>(prec, project, variant, src, dst, d, c, twobeta, err, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gblb
