// Conservation sums without any device allocation.
//
// lb_conserved needs a context, and a context allocates its buffers with
// cudaMalloc.  Some callers cannot allocate: code that runs under a memory
// budget owned by another allocator (a framework's caching allocator that
// holds all device memory), or latency-critical loops that must not pay
// cudaMalloc's implicit device synchronisation.  lb_conserved_noalloc serves
// them: the caller passes the populations and the output, both in its own
// device memory, and the only scratch -- one partial sum per (sub-lattice,
// z) plane -- lives in the file-scope array below, which every GPU that loads
// this library holds until the process exits.
#include <mutex>

#include "gblb.h"
#include "lb_ctx.h"
#include "lb_kernels.cuh"

namespace gblb {

constexpr int kNoAllocMaxPlanes = 4096;  // 2 * nz must not exceed this
constexpr int kNoAllocThreads = 256;

// Scratch shared by every call on a device: slot p holds the five FP64 sums of
// plane p.  Each call writes every slot it reads back, so nothing carries over
// from an earlier call; calls that overlap on the GPU race on these slots.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPlanes * 5];

// One block per (s, z) plane: the plane's nodes in a fixed order (thread t
// takes nodes t, t + 256, ...; then a shared-memory tree).
template <class Codec>
__global__ void __launch_bounds__(kNoAllocThreads) k_conserved_planes(const typename Codec::raw_t* __restrict__ src,
                                                                     Dims d, Consts<typename Codec::R> K,
                                                                     double* __restrict__ partials) {
    using R = typename Codec::R;
    const int plane_id = blockIdx.x;  // s * nz + z
    const int s = plane_id / d.nz, z = plane_id % d.nz;
    const int64_t nxy = (int64_t)d.nx * d.ny;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t k = threadIdx.x; k < nxy; k += kNoAllocThreads) {
        const int64_t q = (int64_t)s * d.plane + (int64_t)z * nxy + k;
        const NodeMoments<R> m = node_moments_at<Codec>(src, d, q, K);
        acc[0] += (double)m.drho;
        acc[1] += (double)m.jx;
        acc[2] += (double)m.jy;
        acc[3] += (double)m.jz;
        acc[4] += (double)m.dk;
    }
    __shared__ double sh[5][kNoAllocThreads];
#pragma unroll
    for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 5; ++c) partials[(int64_t)plane_id * 5 + c] = sh[c][0];
}

// Sum of the plane partials in plane order, then the totals: mass = nodes + sum drho,
// momentum = sum j, energy = (3 theta0 nodes + sum dk) / 2.
__global__ void k_conserved_finish(const double* __restrict__ partials, int nplanes, double nodes, double theta0,
                                   double* __restrict__ out) {
    const int c = threadIdx.x;
    if (c >= 5) return;
    double s = 0.0;
    for (int p = 0; p < nplanes; ++p) s += partials[(int64_t)p * 5 + c];
    if (c == 0)
        out[0] = nodes + s;
    else if (c == 4)
        out[4] = 0.5 * (3.0 * theta0 * nodes + s);
    else
        out[c] = s;
}

}  // namespace gblb

using namespace gblb;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {};
// Error message of the calling host thread's last failed call (errno-style, so that
// threads failing at the same time do not write one string concurrently).
thread_local std::string g_noalloc_msg;
}  // namespace

extern "C" {

lb_status lb_conserved_noalloc(const void* populations, lb_grid grid, lb_precision precision, double* out,
                               void* cuda_stream) {
    if (!populations || !out) {
        g_noalloc_msg = "lb_conserved_noalloc: null pointer";
        return LB_ERR_ARG;
    }
    if (grid.nx < 1 || grid.ny < 1 || grid.nz < 1 || grid.nx > (1 << 30) || grid.ny > (1 << 30)) {
        g_noalloc_msg = "lb_conserved_noalloc: grid extents must be >= 1";
        return LB_ERR_ARG;
    }
    if (2 * grid.nz > kNoAllocMaxPlanes) {
        g_noalloc_msg = "lb_conserved_noalloc: 2 * nz = " + std::to_string(2 * grid.nz) +
                        " planes exceeds the fixed scratch of " + std::to_string(kNoAllocMaxPlanes) + " planes";
        return LB_ERR_ARG;
    }
    if ((int)precision < LB_F64 || (int)precision > LB_F32_S16B) {
        g_noalloc_msg = "lb_conserved_noalloc: unknown precision";
        return LB_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        g_noalloc_msg = std::string("lb_conserved_noalloc: cudaGetDevice: ") + cudaGetErrorString(e);
        return LB_ERR_CUDA;
    }
    double* partials = nullptr;
    {
        // First call on a device, with that device current: look up the device address
        // of the scratch array (the host-side symbol is only a stand-in).
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                g_noalloc_msg = std::string("lb_conserved_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return LB_ERR_CUDA;
            }
            g_partials_ptr[dev] = static_cast<double*>(p);
        }
        partials = g_partials_ptr[dev];
    }
    Dims d;
    d.nx = (int)grid.nx;
    d.ny = (int)grid.ny;
    d.nz = (int)grid.nz;
    d.plane = grid.nx * grid.ny * grid.nz;
    d.rows = 2 * grid.ny * grid.nz;
    const int nplanes = 2 * (int)grid.nz;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const LaunchConsts& lc = lattice_consts();
    switch ((int)precision) {
        case LB_F64:
            k_conserved_planes<CodecF64><<<nplanes, kNoAllocThreads, 0, st>>>(static_cast<const double*>(populations),
                                                                               d, lc.kd, partials);
            break;
        case LB_F32:
            k_conserved_planes<CodecF32><<<nplanes, kNoAllocThreads, 0, st>>>(static_cast<const float*>(populations),
                                                                               d, lc.kf, partials);
            break;
        case LB_F32_S16F:
            k_conserved_planes<CodecF16><<<nplanes, kNoAllocThreads, 0, st>>>(
                static_cast<const __half*>(populations), d, lc.kf, partials);
            break;
        default:
            k_conserved_planes<CodecBF16><<<nplanes, kNoAllocThreads, 0, st>>>(
                static_cast<const __nv_bfloat16*>(populations), d, lc.kf, partials);
            break;
    }
    k_conserved_finish<<<1, 32, 0, st>>>(partials, nplanes, (double)(2 * d.plane), lc.theta0, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_msg = std::string("lb_conserved_noalloc: launch: ") + cudaGetErrorString(e);
        return LB_ERR_CUDA;
    }
    return LB_OK;
}

const char* lb_conserved_noalloc_error(void) { return g_noalloc_msg.c_str(); }

}  // extern "C"
