// FP64 step kernel (parity mode).
#include "lb_kernels.cuh"

namespace gblb {

cudaError_t launch_step_f64(int eq, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                            double twobeta, int* err, cudaStream_t st) {
    const int th = step_threads(d);
    const double* s = static_cast<const double*>(src);
    double* o = static_cast<double*>(dst);
    if (eq == 3)
        k_step<CodecF64, 3><<<step_grid(d, th), th, 0, st>>>(s, o, d, c.kd, twobeta, err);
    else if (eq == 2)
        k_step<CodecF64, 2><<<step_grid(d, th), th, 0, st>>>(s, o, d, c.kd, twobeta, err);
    else if (eq == 1)
        k_step<CodecF64, 1><<<step_grid(d, th), th, 0, st>>>(s, o, d, c.kd, twobeta, err);
    else
        k_step<CodecF64, 0><<<step_grid(d, th), th, 0, st>>>(s, o, d, c.kd, twobeta, err);
    return cudaGetLastError();
}

}  // namespace gblb
