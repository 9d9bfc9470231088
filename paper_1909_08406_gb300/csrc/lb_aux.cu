// Launchers of the non-step kernels: initialisation from fields, node
// moments, global conservation sums and population format conversion.
#include "lb_kernels.cuh"

namespace gblb {

size_t storage_bytes(int prec) {
    switch (prec) {
        case kF64: return 8;
        case kF32: return 4;
        case kF16: return 2;
        case kBF16: return 2;
        default: return 0;
    }
}

template <class Codec>
static const Consts<typename Codec::R>& consts_for(const LaunchConsts& c) {
    if constexpr (std::is_same<typename Codec::R, double>::value)
        return c.kd;
    else
        return c.kf;
}

// Calls f.template operator()<Codec>() for the codec of prec.
template <class F>
static cudaError_t dispatch(int prec, F&& f) {
    switch (prec) {
        case kF64: return f(CodecF64{});
        case kF32: return f(CodecF32{});
        case kF16: return f(CodecF16{});
        case kBF16: return f(CodecBF16{});
        default: return cudaErrorInvalidValue;
    }
}

static unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

cudaError_t launch_step(int prec, int eq, int variant, const void* src, void* dst, const Dims& d,
                        const LaunchConsts& c, double twobeta, int* err, cudaStream_t st) {
    if (prec == kF64) return launch_step_f64(eq, src, dst, d, c, twobeta, err, st);
    if (eq >= 2) return launch_step_entropic(prec, eq, src, dst, d, c, twobeta, err, st);
    return launch_step_f32(prec, eq == 1, variant, src, dst, d, c, twobeta, err, st);
}

cudaError_t launch_init(int prec, int eq, void* dst, const Dims& d, const LaunchConsts& c, int64_t q0,
                        int64_t count, const double* rho, const double* u, int64_t ustride, const double* theta,
                        int* err, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    return dispatch(prec, [&](auto codec) {
        using C = decltype(codec);
        using T = typename C::raw_t;
        const unsigned nb = blocks_for(count, 256);
        T* o = static_cast<T*>(dst);
        if (eq >= 2)  // the exact entropic equilibrium (kind 3 adds only the path length)
            k_init<C, 2><<<nb, 256, 0, st>>>(o, d, consts_for<C>(c), c.theta0, q0, count, rho, u, ustride, theta, err);
        else if (eq == 1)
            k_init<C, 1><<<nb, 256, 0, st>>>(o, d, consts_for<C>(c), c.theta0, q0, count, rho, u, ustride, theta, err);
        else
            k_init<C, 0><<<nb, 256, 0, st>>>(o, d, consts_for<C>(c), c.theta0, q0, count, rho, u, ustride, theta, err);
        return cudaGetLastError();
    });
}

cudaError_t launch_moments(int prec, const void* src, const Dims& d, const LaunchConsts& c, int64_t q0, int64_t count,
                           double* rho, double* u, int64_t ustride, double* theta, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    return dispatch(prec, [&](auto codec) {
        using C = decltype(codec);
        using T = typename C::raw_t;
        k_moments<C><<<blocks_for(count, 256), 256, 0, st>>>(static_cast<const T*>(src), d, consts_for<C>(c), c.theta0,
                                                              q0, count, rho, u, ustride, theta);
        return cudaGetLastError();
    });
}

// Sum of the per-block partials in a fixed order: thread t adds blocks
// t, t + 256, ... then a shared-memory tree.
__global__ void __launch_bounds__(kRedThreads) k_reduce_partials(const double* __restrict__ partials, int nblocks,
                                                                  double* __restrict__ out5) {
    __shared__ double sh[5][kRedThreads];
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kRedThreads)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += partials[(int64_t)b * 5 + k];
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) out5[k] = sh[k][0];
}

cudaError_t launch_conserved(int prec, const void* src, const Dims& d, const LaunchConsts& c, double* partials,
                             int nblocks, double* out5, cudaStream_t st, int64_t z0, int64_t nzr) {
    if (nzr < 0) nzr = d.nz;
    cudaError_t e = dispatch(prec, [&](auto codec) {
        using C = decltype(codec);
        using T = typename C::raw_t;
        k_conserved<C><<<nblocks, kRedThreads, 0, st>>>(static_cast<const T*>(src), d, consts_for<C>(c), partials, z0,
                                                         nzr);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    k_reduce_partials<<<1, kRedThreads, 0, st>>>(partials, nblocks, out5);
    return cudaGetLastError();
}

// blockIdx.y = entry k of the list, blockIdx.z = sub-lattice s, x over the plane's ny nx elements.
template <class T>
__global__ void __launch_bounds__(256) k_halo_copy(T* __restrict__ f, Dims d, HaloList list, T* __restrict__ buf,
                                                   int pack) {
    const int k = blockIdx.y, s = blockIdx.z;
    const int64_t nxy = (int64_t)d.nx * d.ny;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nxy) return;
    T* a = f + ((int64_t)s * kQ + list.pop[k]) * d.plane + (int64_t)list.plane[k] * nxy + e;
    T* b = buf + ((int64_t)k * 2 + s) * nxy + e;
    if (pack)
        *b = *a;
    else
        *a = *b;
}

cudaError_t launch_halo_copy(int prec, void* f, const Dims& d, const HaloList& list, void* buf, bool pack,
                             cudaStream_t st) {
    if (list.n <= 0) return cudaSuccess;
    const int64_t nxy = (int64_t)d.nx * d.ny;
    const dim3 grid(blocks_for(nxy, 256), (unsigned)list.n, 2);
    switch (storage_bytes(prec)) {
        case 8: k_halo_copy<uint64_t><<<grid, 256, 0, st>>>(static_cast<uint64_t*>(f), d, list, static_cast<uint64_t*>(buf), pack); break;
        case 4: k_halo_copy<uint32_t><<<grid, 256, 0, st>>>(static_cast<uint32_t*>(f), d, list, static_cast<uint32_t*>(buf), pack); break;
        case 2: k_halo_copy<uint16_t><<<grid, 256, 0, st>>>(static_cast<uint16_t*>(f), d, list, static_cast<uint16_t*>(buf), pack); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_to_f64(int prec, const void* src, const Dims& d, const LaunchConsts& c, int64_t e0, int64_t count,
                          double* f, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    return dispatch(prec, [&](auto codec) {
        using C = decltype(codec);
        using T = typename C::raw_t;
        k_to_f64<C><<<blocks_for(count, 256), 256, 0, st>>>(static_cast<const T*>(src), d.plane, c.w41, e0, count, f);
        return cudaGetLastError();
    });
}

cudaError_t launch_from_f64(int prec, const double* f, void* dst, const Dims& d, const LaunchConsts& c, int64_t e0,
                            int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    return dispatch(prec, [&](auto codec) {
        using C = decltype(codec);
        using T = typename C::raw_t;
        k_from_f64<C><<<blocks_for(count, 256), 256, 0, st>>>(f, d.plane, c.w41, e0, count, static_cast<T*>(dst));
        return cudaGetLastError();
    });
}

}  // namespace gblb
