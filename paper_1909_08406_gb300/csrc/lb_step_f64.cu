// FP64 step kernel (parity mode).
#include "lb_kernels.cuh"

namespace gblb {

cudaError_t launch_step_f64(bool project, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                            double twobeta, int* err, cudaStream_t st) {
    const int th = step_threads(d);
    const double* s = static_cast<const double*>(src);
    double* o = static_cast<double*>(dst);
    if (project)
        k_step<CodecF64, true><<<step_grid(d, th), th, 0, st>>>(s, o, d, c.kd, twobeta, err);
    else
        k_step<CodecF64, false><<<step_grid(d, th), th, 0, st>>>(s, o, d, c.kd, twobeta, err);
    return cudaGetLastError();
}

}  // namespace gblb
