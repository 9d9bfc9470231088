// The update with the exact entropic equilibrium (Eqs. (discreteentropiceq),
// (fivelagrangemultipliersystem)): k_step with a per-node Newton solve of the
// five Lagrange multipliers, FP32 arithmetic for FP32/FP16/BF16 storage.
// eq 3: with the entropic path length (entropic_path).  (The FP64 mode instantiates the same
// kernel in lb_step_f64.cu.)
#include "lb_kernels.cuh"

namespace gblb {

cudaError_t launch_step_entropic(int prec, int eq, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                                 double twobeta, int* err, cudaStream_t st) {
    const int th = step_threads(d);
    auto run = [&](auto codec) {
        using C = decltype(codec);
        using T = typename C::raw_t;
        if (eq == 3)
            k_step<C, 3><<<step_grid(d, th), th, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                          (float)twobeta, err);
        else
            k_step<C, 2><<<step_grid(d, th), th, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), d, c.kf,
                                                          (float)twobeta, err);
        return cudaGetLastError();
    };
    switch (prec) {
        case kF32: return run(CodecF32{});
        case kF16: return run(CodecF16{});
        case kBF16: return run(CodecBF16{});
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gblb
