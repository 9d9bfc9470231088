// FP32-arithmetic step kernels (FP32, FP16 and BF16 storage).  This unit is
// compiled with ptxas double-precision-use warnings so that no FP64
// instruction slips into the float path.
#include "lb_kernels.cuh"

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

cudaError_t launch_step_f32(int prec, bool project, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                            double twobeta, int* err, cudaStream_t st) {
    switch (prec) {
        case kF32:
            return project ? run<CodecF32, true>(src, dst, d, c, twobeta, err, st)
                           : run<CodecF32, false>(src, dst, d, c, twobeta, err, st);
        case kF16:
            return project ? run<CodecF16, true>(src, dst, d, c, twobeta, err, st)
                           : run<CodecF16, false>(src, dst, d, c, twobeta, err, st);
        case kBF16:
            return project ? run<CodecBF16, true>(src, dst, d, c, twobeta, err, st)
                           : run<CodecBF16, false>(src, dst, d, c, twobeta, err, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace gblb
