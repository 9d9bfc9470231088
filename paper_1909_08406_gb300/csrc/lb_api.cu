// C ABI of the RD3Q41 solver (declared in include/gblb.h): context
// management, host/device transfers and the time-step loop.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gblb.h"
#include "lb_ctx.h"
#include "lb_launch.h"

using namespace gblb;

// Table I of the paper (Sec. IV): weight of one velocity of each moving shell.
static const double kTableI[5] = {
    0.04743040745116578,  // sc-1
    0.00165687664501576,  // sc-2
    0.00651175327832464,  // fcc-1
    0.00454087801154440,  // bcc-1
    0.04917980624482672,  // bcc-1/2
};

struct Lattice {
    LaunchConsts lc;
    double theta0;
};


// Lattice constants from Table I.  w_0 = 1 - sum of the other weights and
// theta_0 = sum_i w_i c_ix^2 (Sec. III, Eq. allWeights).  The rest-state
// equilibrium polynomial (Sec. V) per shell: with s = c^2/theta_0,
//   f~/(w rho) = 1 + eta (s-3)/2 + eta^2 (s^2-10s+15)/8 + eta^3 (s^3-21s^2+105s-105)/48.
// M_2 = <f~, c^2 c_x^2>/(5 rho theta^2) - 1 and M_2' = <f~, c_x^2 c_y^2>/(rho theta^2) - 1
// are cubic polynomials in eta divided by (1+eta)^2; their coefficients are
// summed here exactly over the lattice, once, in FP64.
static Lattice make_lattice() {
    Lattice L;
    double w41[kQ];
    double sum = 0.0;
    for (int i = 1; i < kQ; ++i) {
        w41[i] = kTableI[vel(i).shell - 1];
        sum += w41[i];
    }
    w41[0] = 1.0 - sum;
    double th0 = 0.0;
    for (int i = 0; i < kQ; ++i) th0 += w41[i] * (0.5 * vel(i).x) * (0.5 * vel(i).x);
    L.theta0 = th0;
    Consts<double> k;
    memset(&k, 0, sizeof k);
    double pk[kShells][4];
    for (int s = 0; s < kShells; ++s) {
        int first = -1;
        for (int i = 0; i < kQ; ++i)
            if (vel(i).shell == s && first < 0) first = i;
        const Vel c = vel(first);
        const double csq = 0.25 * (c.x * c.x + c.y * c.y + c.z * c.z);
        const double st = csq / th0;
        k.w[s] = w41[first];
        k.c2[s] = csq;
        k.p1[s] = 0.5 * (st - 3.0);
        k.p2[s] = (st * st - 10.0 * st + 15.0) / 8.0;
        k.p3[s] = (st * st * st - 21.0 * st * st + 105.0 * st - 105.0) / 48.0;
        pk[s][0] = 1.0;
        pk[s][1] = k.p1[s];
        pk[s][2] = k.p2[s];
        pk[s][3] = k.p3[s];
        for (int i = 0; i < kQ; ++i) {
            if (vel(i).shell != s) continue;
            const double cx = 0.5 * vel(i).x, cy = 0.5 * vel(i).y;
            k.n2[s] += cx * cx;
            k.n4[s] += cx * cx * cx * cx;
            k.n22[s] += cx * cx * cy * cy;
        }
        // the projection's shell sums folded into cubics in eta
        for (int p = 0; p < 4; ++p) {
            k.pj[0][p] += k.w[s] * k.n2[s] * pk[s][p];
            k.pj[1][p] += k.w[s] * k.n2[s] * csq * pk[s][p];
            k.pj[2][p] += k.w[s] * k.n4[s] * pk[s][p];
            k.pj[3][p] += k.w[s] * k.n22[s] * pk[s][p];
        }
    }
    double A[4] = {0, 0, 0, 0}, B[4] = {0, 0, 0, 0};
    for (int i = 0; i < kQ; ++i) {
        const Vel c = vel(i);
        const double cx = 0.5 * c.x, cy = 0.5 * c.y, cz = 0.5 * c.z;
        const double csq = cx * cx + cy * cy + cz * cz;
        for (int p = 0; p < 4; ++p) {
            A[p] += w41[i] * csq * cx * cx * pk[c.shell][p];
            B[p] += w41[i] * cx * cx * cy * cy * pk[c.shell][p];
        }
    }
    const double t2 = th0 * th0;
    const double one_two_one[4] = {1.0, 2.0, 1.0, 0.0};  // (1 + eta)^2
    for (int p = 0; p < 4; ++p) {
        k.m2[p] = A[p] / (5.0 * t2) - one_two_one[p];
        k.m2p[p] = B[p] / t2 - one_two_one[p];
    }
    k.theta0 = th0;
    k.inv_3theta0 = 1.0 / (3.0 * th0);
    L.lc.kd = k;
    Consts<float>& f = L.lc.kf;
    for (int s = 0; s < kShells; ++s) {
        f.w[s] = (float)k.w[s];
        f.c2[s] = (float)k.c2[s];
        f.p1[s] = (float)k.p1[s];
        f.p2[s] = (float)k.p2[s];
        f.p3[s] = (float)k.p3[s];
        f.n2[s] = (float)k.n2[s];
        f.n4[s] = (float)k.n4[s];
        f.n22[s] = (float)k.n22[s];
    }
    for (int j = 0; j < 4; ++j)
        for (int p = 0; p < 4; ++p) f.pj[j][p] = (float)k.pj[j][p];
    for (int p = 0; p < 4; ++p) {
        f.m2[p] = (float)k.m2[p];
        f.m2p[p] = (float)k.m2p[p];
    }
    f.theta0 = (float)th0;
    f.inv_3theta0 = (float)(1.0 / (3.0 * th0));
    for (int i = 0; i < kQ; ++i) L.lc.w41.w[i] = w41[i];
    L.lc.theta0 = th0;
    return L;
}

static const Lattice& lattice() {
    static const Lattice L = make_lattice();
    return L;
}

namespace gblb {
const LaunchConsts& lattice_consts() { return lattice().lc; }
}  // namespace gblb

static std::string g_init_msg;

static lb_status fail(lb_ctx* c, lb_status s, const std::string& m) {
    if (c)
        c->msg = m;
    else
        g_init_msg = m;
    return s;
}

#define CK(ctx, call)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    } while (0)

static int64_t nodes_of(const lb_ctx* c) { return 2 * c->d.plane; }

// Device address of a host array that kernels can read and write directly: page-locked
// (pinned) host memory, mapped into the device's address space.  nullptr for pageable memory,
// which goes through the staging buffer instead.
static const void* mapped_host_view(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error of an unknown pointer
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// True for device memory (or managed memory) the kernels can write.
static bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Staging buffer for host transfers (float64), allocated on first use.
static lb_status ensure_stage(lb_ctx* c) {
    if (c->d_stage) return LB_OK;
    const int64_t total = 2 * kQ * c->d.plane;
    int64_t want = (int64_t)1 << 26;  // 64 Mi doubles = 512 MiB
    if (want > total) want = total;
    if (want < 5) want = 5;
    CK(c, cudaMalloc(&c->d_stage, (size_t)want * sizeof(double)));
    c->stage_doubles = want;
    return LB_OK;
}

extern "C" {

lb_status lb_velocity_set(int* c2, double* w) {
    const Lattice& L = lattice();
    for (int i = 0; i < kQ; ++i) {
        if (c2) {
            c2[3 * i + 0] = vel(i).x;
            c2[3 * i + 1] = vel(i).y;
            c2[3 * i + 2] = vel(i).z;
        }
        if (w) w[i] = L.lc.w41.w[i];
    }
    return LB_OK;
}

double lb_theta0(void) { return lattice().theta0; }

lb_status lb_init(lb_ctx** out, lb_grid grid, int velocity_set, double theta0, double tau, lb_precision precision,
                  unsigned flags, void* cuda_stream) {
    if (!out) return fail(nullptr, LB_ERR_ARG, "lb_init: out is NULL");
    *out = nullptr;
    if (velocity_set != LB_RD3Q41) return fail(nullptr, LB_ERR_ARG, "lb_init: only the RD3Q41 velocity set exists");
    if (grid.nx < 1 || grid.ny < 1 || grid.nz < 1 || grid.nx > (1 << 30) || grid.ny > (1 << 30) ||
        grid.nz > (1 << 30))
        return fail(nullptr, LB_ERR_ARG, "lb_init: grid extents must be in [1, 2^30]");
    if (2 * grid.ny * grid.nz > 0x7fffffffLL || (grid.nx + 127) / 128 > 65535)
        return fail(nullptr, LB_ERR_ARG, "lb_init: grid too large for the launch geometry");
    if (grid.nx * grid.ny > ((int64_t)1 << 40) / grid.nz)
        return fail(nullptr, LB_ERR_ARG, "lb_init: more than 2^40 cells");
    if ((int)precision < LB_F64 || (int)precision > LB_F32_S16B)
        return fail(nullptr, LB_ERR_ARG, "lb_init: unknown precision");
    if (!(tau > 0.0)) return fail(nullptr, LB_ERR_ARG, "lb_init: tau must be > 0 (or +inf)");
    if (flags & ~(LB_FLAG_PAPER_LITERAL | LB_FLAG_STAGED | LB_FLAG_ENTROPIC | LB_FLAG_ENTROPIC_PATH))
        return fail(nullptr, LB_ERR_ARG, "lb_init: unknown flag bits");
    if ((flags & LB_FLAG_ENTROPIC) && (flags & LB_FLAG_PAPER_LITERAL))
        return fail(nullptr, LB_ERR_ARG, "lb_init: LB_FLAG_ENTROPIC and LB_FLAG_PAPER_LITERAL exclude each other");
    if ((flags & LB_FLAG_ENTROPIC_PATH) && !(flags & LB_FLAG_ENTROPIC))
        return fail(nullptr, LB_ERR_ARG, "lb_init: LB_FLAG_ENTROPIC_PATH needs LB_FLAG_ENTROPIC");
    const Lattice& L = lattice();
    if (theta0 > 0.0 && fabs(theta0 / L.theta0 - 1.0) > 1e-12)
        return fail(nullptr, LB_ERR_THETA0, "lb_init: theta0 differs from sum_i w_i c_ix^2 of the Table I weights");

    lb_ctx* c = new lb_ctx();
    c->g = grid;
    c->d.nx = (int)grid.nx;
    c->d.ny = (int)grid.ny;
    c->d.nz = (int)grid.nz;
    c->d.plane = grid.nx * grid.ny * grid.nz;
    c->d.rows = 2 * grid.ny * grid.nz;
    c->prec = (int)precision;
    c->eq = (flags & LB_FLAG_ENTROPIC) ? ((flags & LB_FLAG_ENTROPIC_PATH) ? 3 : 2) : (flags & LB_FLAG_PAPER_LITERAL) ? 0 : 1;
    c->variant = (flags & LB_FLAG_STAGED) ? kKernelStaged : kKernelAuto;
    c->tau = tau;
    c->twobeta = isinf(tau) ? 0.0 : 2.0 / (2.0 * tau + 1.0);
    c->stream = (cudaStream_t)cuda_stream;
    c->esize = storage_bytes(c->prec);
    c->cur = 0;
    c->time = 0;
    cudaError_t e = cudaGetDevice(&c->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, LB_ERR_CUDA, std::string("lb_init: ") + cudaGetErrorString(e));
    }
    c->nblocks = sms > 0 ? 4 * sms : 256;
    const size_t bytes = (size_t)(2 * kQ) * (size_t)c->d.plane * c->esize;
    void* p[2] = {nullptr, nullptr};
    int* err = nullptr;
    double* part = nullptr;
    e = cudaMalloc(&p[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)(c->nblocks * 5 + 5) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(p[0], 0, bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p[1], 0, bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(p[0]);
        cudaFree(p[1]);
        cudaFree(err);
        cudaFree(part);
        delete c;
        cudaGetLastError();
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,
                    std::string("lb_init: ") + cudaGetErrorString(e));
    }
    c->buf[0] = p[0];
    c->buf[1] = p[1];
    c->d_err = err;
    c->d_partials = part;
    c->d_out5 = part + c->nblocks * 5;
    *out = c;
    return LB_OK;
}

lb_status lb_set_stream(lb_ctx* c, void* cuda_stream) {
    if (!c) return LB_ERR_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return LB_OK;
}

lb_status lb_sync(lb_ctx* c) {
    if (!c) return LB_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaStreamSynchronize(c->stream));
    int h = 0;
    CK(c, cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & 2) return fail(c, LB_ERR_TIMEOUT, "a bounded wait in the staged step kernel gave up");
    if (h) return fail(c, LB_ERR_UNSTABLE, "a node reached rho <= 0, theta <= 0 or a non-finite moment");
    return LB_OK;
}

int lb_step_variant(const lb_ctx* c) {
    if (!c) return -1;
    if (c->eq >= 2) return kKernelDirect1;  // the exact entropic equilibrium runs in k_step only
    if (c->sr)  // the stochastic store: the x-pair kernel where it applies, else one node per thread
        return resolve_kernel(c->prec, c->d, kKernelDirect2XL) == kKernelDirect2XL ? kKernelDirect2XL : kKernelDirect1;
    return resolve_kernel(c->prec, c->d, c->variant);
}

lb_status lb_set_step_kernel(lb_ctx* c, int kernel) {
    if (!c || kernel < LB_KERNEL_AUTO || kernel > LB_KERNEL_DIRECT2XL) return fail(c, LB_ERR_ARG, "lb_set_step_kernel: unknown kernel");
    c->variant = kernel;
    return LB_OK;
}

lb_status lb_tune(lb_ctx* c, int reps, int* kernel_out, double* ms_out) {
    if (!c) return LB_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    if (reps < 1) reps = 3;
    const LaunchConsts& lc = lattice().lc;
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_k = resolve_kernel(c->prec, c->d, kKernelAuto);
    // trial steps read buf[cur] and write buf[1 - cur] without flipping: the state is unchanged
    for (int k = LB_KERNEL_DIRECT1; k <= LB_KERNEL_DIRECT2XL; ++k) {
        if (resolve_kernel(c->prec, c->d, k) != k) continue;
        cudaError_t e = launch_step(c->prec, c->eq, k, c->buf[c->cur], c->buf[1 - c->cur], c->d, lc, c->twobeta,
                                    c->d_err, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = launch_step(c->prec, c->eq, k, c->buf[c->cur], c->buf[1 - c->cur], c->d, lc, c->twobeta, c->d_err,
                            c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(c, LB_ERR_CUDA, std::string("lb_tune: ") + cudaGetErrorString(e));
        }
        ms /= reps;
        if (ms < best) {
            best = ms;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->variant = best_k;
    if (kernel_out) *kernel_out = best_k;
    if (ms_out) *ms_out = best;
    return LB_OK;
}

lb_status lb_set_fields(lb_ctx* c, const double* rho, const double* u, const double* theta, int on_device) {
    if (!c || !rho || !u || !theta) return fail(c, LB_ERR_ARG, "lb_set_fields: null argument");
    CK(c, cudaSetDevice(c->device));
    const int64_t n = nodes_of(c);
    const LaunchConsts& lc = lattice().lc;
    void* dst = c->buf[c->cur];
    const double* mr = on_device ? nullptr : static_cast<const double*>(mapped_host_view(rho));
    const double* mu = on_device ? nullptr : static_cast<const double*>(mapped_host_view(u));
    const double* mt = on_device ? nullptr : static_cast<const double*>(mapped_host_view(theta));
    if (on_device) {
        CK(c, launch_init(c->prec, c->eq, dst, c->d, lc, 0, n, rho, u, n, theta, c->d_err, c->stream));
    } else if (mr && mu && mt) {
        // pinned host arrays: the kernel reads them over the host link, no staging copies
        CK(c, launch_init(c->prec, c->eq, dst, c->d, lc, 0, n, mr, mu, n, mt, c->d_err, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    } else {
        lb_status s = ensure_stage(c);
        if (s != LB_OK) return s;
        const int64_t chunk = c->stage_doubles / 5;
        for (int64_t q0 = 0; q0 < n; q0 += chunk) {
            const int64_t cnt = n - q0 < chunk ? n - q0 : chunk;
            double* sr = c->d_stage;
            double* su = sr + cnt;
            double* st = su + 3 * cnt;
            const size_t b = (size_t)cnt * sizeof(double);
            CK(c, cudaMemcpyAsync(sr, rho + q0, b, cudaMemcpyHostToDevice, c->stream));
            for (int k = 0; k < 3; ++k)
                CK(c, cudaMemcpyAsync(su + k * cnt, u + k * n + q0, b, cudaMemcpyHostToDevice, c->stream));
            CK(c, cudaMemcpyAsync(st, theta + q0, b, cudaMemcpyHostToDevice, c->stream));
            CK(c, launch_init(c->prec, c->eq, dst, c->d, lc, q0, cnt, sr, su, cnt, st, c->d_err, c->stream));
        }
        CK(c, cudaStreamSynchronize(c->stream));
    }
    c->time = 0;
    return LB_OK;
}

lb_status lb_step(lb_ctx* c, int64_t n) {
    if (!c || n < 0) return fail(c, LB_ERR_ARG, "lb_step: bad argument");
    CK(c, cudaSetDevice(c->device));
    const LaunchConsts& lc = lattice().lc;
    for (int64_t t = 0; t < n; ++t) {
        if (c->nonideal)
            CK(c, launch_nonideal_step(c->prec, c->buf[c->cur], c->buf[1 - c->cur], c->d, lc, c->twobeta,
                                       c->nonideal, c->ni_eos, c->d_ni, c->d_err, c->stream));
        else if (c->sr)
            CK(c, launch_step_sr(c->buf[c->cur], c->buf[1 - c->cur], c->d, lc, c->twobeta, c->d_err, c->stream,
                                 sr_step_key(c->sr_seed, c->sr_t++)));
        else if (c->walls)
            CK(c, launch_wall_step(c->prec, c->eq, c->variant, c->buf[c->cur], c->buf[1 - c->cur], c->d, lc,
                                   c->twobeta, c->d_wall, c->d_err, c->stream));
        else
            CK(c, launch_step(c->prec, c->eq, c->variant, c->buf[c->cur], c->buf[1 - c->cur], c->d, lc,
                              c->twobeta, c->d_err, c->stream));
        c->cur ^= 1;
        c->time += 1;
    }
    return LB_OK;
}

lb_status lb_get_moments(lb_ctx* c, double* rho, double* u, double* theta, int on_device) {
    if (!c) return LB_ERR_ARG;
    CK(c, cudaSetDevice(c->device));
    const int64_t n = nodes_of(c);
    const LaunchConsts& lc = lattice().lc;
    const void* src = c->buf[c->cur];
    if (on_device) {
        CK(c, launch_moments(c->prec, src, c->d, lc, 0, n, rho, u, n, theta, c->stream));
        return LB_OK;
    }
    {
        // pinned host arrays (every one that is requested): the kernel writes them directly
        double* mr = static_cast<double*>(const_cast<void*>(mapped_host_view(rho)));
        double* mu = static_cast<double*>(const_cast<void*>(mapped_host_view(u)));
        double* mt = static_cast<double*>(const_cast<void*>(mapped_host_view(theta)));
        if ((!rho || mr) && (!u || mu) && (!theta || mt)) {
            CK(c, launch_moments(c->prec, src, c->d, lc, 0, n, mr, mu, n, mt, c->stream));
            return lb_sync(c);
        }
    }
    lb_status s = ensure_stage(c);
    if (s != LB_OK) return s;
    const int64_t chunk = c->stage_doubles / 5;
    for (int64_t q0 = 0; q0 < n; q0 += chunk) {
        const int64_t cnt = n - q0 < chunk ? n - q0 : chunk;
        double* sr = c->d_stage;
        double* su = sr + cnt;
        double* st = su + 3 * cnt;
        const size_t b = (size_t)cnt * sizeof(double);
        CK(c, launch_moments(c->prec, src, c->d, lc, q0, cnt, rho ? sr : nullptr, u ? su : nullptr, cnt,
                             theta ? st : nullptr, c->stream));
        if (rho) CK(c, cudaMemcpyAsync(rho + q0, sr, b, cudaMemcpyDeviceToHost, c->stream));
        if (u)
            for (int k = 0; k < 3; ++k)
                CK(c, cudaMemcpyAsync(u + k * n + q0, su + k * cnt, b, cudaMemcpyDeviceToHost, c->stream));
        if (theta) CK(c, cudaMemcpyAsync(theta + q0, st, b, cudaMemcpyDeviceToHost, c->stream));
    }
    return lb_sync(c);
}

lb_status lb_conserved(lb_ctx* c, double out[5]) {
    if (!c || !out) return fail(c, LB_ERR_ARG, "lb_conserved: null argument");
    CK(c, cudaSetDevice(c->device));
    const LaunchConsts& lc = lattice().lc;
    CK(c, launch_conserved(c->prec, c->buf[c->cur], c->d, lc, c->d_partials, c->nblocks, c->d_out5, c->stream));
    double s[5];
    CK(c, cudaMemcpyAsync(s, c->d_out5, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    lb_status st = lb_sync(c);
    if (st != LB_OK) return st;
    const double n = (double)nodes_of(c);
    out[0] = n + s[0];
    out[1] = s[1];
    out[2] = s[2];
    out[3] = s[3];
    out[4] = 0.5 * (3.0 * lattice().theta0 * n + s[4]);
    return LB_OK;
}

lb_status lb_conserved_planes(lb_ctx* c, int64_t z0, int64_t z1, double out[5]) {
    if (!c || !out) return fail(c, LB_ERR_ARG, "lb_conserved_planes: null argument");
    if (z0 < 0 || z1 > c->d.nz || z0 >= z1) return fail(c, LB_ERR_ARG, "lb_conserved_planes: need 0 <= z0 < z1 <= nz");
    CK(c, cudaSetDevice(c->device));
    const LaunchConsts& lc = lattice().lc;
    CK(c, launch_conserved(c->prec, c->buf[c->cur], c->d, lc, c->d_partials, c->nblocks, c->d_out5, c->stream, z0,
                           z1 - z0));
    double s[5];
    CK(c, cudaMemcpyAsync(s, c->d_out5, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    lb_status st = lb_sync(c);
    if (st != LB_OK) return st;
    const double n = 2.0 * (double)(z1 - z0) * (double)c->d.nx * (double)c->d.ny;
    out[0] = n + s[0];
    out[1] = s[1];
    out[2] = s[2];
    out[3] = s[3];
    out[4] = 0.5 * (3.0 * lattice().theta0 * n + s[4]);
    return LB_OK;
}

// The (plane, population) entries of one halo message of a padded slab of nzp planes (LB_HALO
// halo planes at each end).  An interior node pulls population i from ceil(|c_iz|) cells away at
// most, so the halo plane at distance d from the interior is read only through the populations
// with c_z pointing into the slab and (|2 c_z| + 1) / 2 >= d.  Entries run d = 1, 2, populations
// ascending.  pack: the interior planes a neighbour's halo receives (side 0: the bottom ones, for
// rank - 1's upper halo; side 1: the top ones, for rank + 1's lower halo); unpack: this slab's
// halo (side 0: lower, from rank - 1; side 1: upper, from rank + 1).
static HaloList halo_list(int nzp, int side, bool pack) {
    HaloList L{};
    L.n = 0;
    // populations arriving through the lower halo have c_z > 0, through the upper one c_z < 0
    const bool up = pack ? side == 1 : side == 0;
    for (int dist = 1; dist <= LB_HALO; ++dist) {
        int plane;
        if (pack)
            plane = side == 1 ? nzp - LB_HALO - dist : LB_HALO + dist - 1;
        else
            plane = side == 0 ? LB_HALO - dist : nzp - LB_HALO + dist - 1;
        for (int i = 0; i < kQ; ++i) {
            const int cz2 = vel(i).z;
            const int reach = ((cz2 < 0 ? -cz2 : cz2) + 1) / 2;
            if ((up ? cz2 > 0 : cz2 < 0) && reach >= dist) {
                L.plane[L.n] = plane;
                L.pop[L.n] = i;
                ++L.n;
            }
        }
    }
    return L;
}

static bool halo_ok(lb_ctx* c, const char* who) {
    if (c->d.nz < 3 * LB_HALO) {
        fail(c, LB_ERR_ARG, std::string(who) + ": a padded slab has at least 3 LB_HALO planes");
        return false;
    }
    return true;
}

lb_status lb_halo_bytes(lb_ctx* c, int64_t* bytes) {
    if (!c || !bytes) return fail(c, LB_ERR_ARG, "lb_halo_bytes: null argument");
    if (!halo_ok(c, "lb_halo_bytes")) return LB_ERR_ARG;
    const HaloList L = halo_list(c->d.nz, 0, true);
    *bytes = (int64_t)L.n * 2 * c->d.nx * c->d.ny * (int64_t)c->esize;
    return LB_OK;
}

static lb_status halo_copy(lb_ctx* c, int side, void* buf, bool pack, const char* who) {
    if (!c || !buf || (side != 0 && side != 1)) return fail(c, LB_ERR_ARG, std::string(who) + ": bad argument");
    if (!halo_ok(c, who)) return LB_ERR_ARG;
    if (!is_device_pointer(buf)) return fail(c, LB_ERR_ARG, std::string(who) + ": the buffer must be device memory");
    CK(c, cudaSetDevice(c->device));
    CK(c, launch_halo_copy(c->prec, c->buf[c->cur], c->d, halo_list(c->d.nz, side, pack), buf, pack, c->stream));
    return LB_OK;
}

lb_status lb_halo_pack(lb_ctx* c, int side, void* buf) { return halo_copy(c, side, buf, true, "lb_halo_pack"); }

lb_status lb_halo_unpack(lb_ctx* c, int side, const void* buf) {
    return halo_copy(c, side, const_cast<void*>(buf), false, "lb_halo_unpack");
}

lb_status lb_get_populations(lb_ctx* c, double* f, int on_device) {
    if (!c || !f) return fail(c, LB_ERR_ARG, "lb_get_populations: null argument");
    CK(c, cudaSetDevice(c->device));
    const int64_t total = 2 * kQ * c->d.plane;
    const LaunchConsts& lc = lattice().lc;
    const void* src = c->buf[c->cur];
    if (on_device) {
        CK(c, launch_to_f64(c->prec, src, c->d, lc, 0, total, f, c->stream));
        return LB_OK;
    }
    lb_status s = ensure_stage(c);
    if (s != LB_OK) return s;
    for (int64_t e0 = 0; e0 < total; e0 += c->stage_doubles) {
        const int64_t cnt = total - e0 < c->stage_doubles ? total - e0 : c->stage_doubles;
        CK(c, launch_to_f64(c->prec, src, c->d, lc, e0, cnt, c->d_stage, c->stream));
        CK(c, cudaMemcpyAsync(f + e0, c->d_stage, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    return lb_sync(c);
}

lb_status lb_set_populations(lb_ctx* c, const double* f, int on_device) {
    if (!c || !f) return fail(c, LB_ERR_ARG, "lb_set_populations: null argument");
    CK(c, cudaSetDevice(c->device));
    const int64_t total = 2 * kQ * c->d.plane;
    const LaunchConsts& lc = lattice().lc;
    void* dst = c->buf[c->cur];
    if (on_device) {
        CK(c, launch_from_f64(c->prec, f, dst, c->d, lc, 0, total, c->stream));
    } else {
        lb_status s = ensure_stage(c);
        if (s != LB_OK) return s;
        for (int64_t e0 = 0; e0 < total; e0 += c->stage_doubles) {
            const int64_t cnt = total - e0 < c->stage_doubles ? total - e0 : c->stage_doubles;
            CK(c, cudaMemcpyAsync(c->d_stage, f + e0, (size_t)cnt * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream));
            CK(c, launch_from_f64(c->prec, c->d_stage, dst, c->d, lc, e0, cnt, c->stream));
        }
        CK(c, cudaStreamSynchronize(c->stream));
    }
    c->time = 0;
    return LB_OK;
}

int64_t lb_state_bytes(const lb_ctx* c) { return c ? (int64_t)(2 * kQ) * c->d.plane * (int64_t)c->esize : -1; }

lb_status lb_get_grid(const lb_ctx* c, lb_grid* grid) {
    if (!c || !grid) return LB_ERR_ARG;
    *grid = c->g;
    return LB_OK;
}

lb_status lb_get_state(lb_ctx* c, void* raw, int on_device) {
    if (!c || !raw) return fail(c, LB_ERR_ARG, "lb_get_state: null argument");
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaMemcpyAsync(raw, c->buf[c->cur], (size_t)lb_state_bytes(c),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (on_device) return LB_OK;
    return lb_sync(c);
}

lb_status lb_set_state(lb_ctx* c, const void* raw, int on_device) {
    if (!c || !raw) return fail(c, LB_ERR_ARG, "lb_set_state: null argument");
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaMemcpyAsync(c->buf[c->cur], raw, (size_t)lb_state_bytes(c),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
    c->time = 0;
    return LB_OK;
}

int64_t lb_time(const lb_ctx* c) { return c ? c->time : -1; }

lb_status lb_destroy(lb_ctx* c) {
    if (!c) return LB_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->buf[0]);
    cudaFree(c->buf[1]);
    cudaFree(c->d_err);
    cudaFree(c->d_partials);
    cudaFree(c->d_stage);
    cudaFree(c->d_wall);
    cudaFree(c->d_ni);
    delete c;
    return LB_OK;
}

// Upload per-column wall parameters ([2][3][ncol] doubles, host) and derive the walls.
static lb_status set_wall_columns(lb_ctx* c, const double* params) {
    const int64_t ncol = (int64_t)c->d.nx * c->d.ny;
    CK(c, cudaSetDevice(c->device));
    if (!c->d_wall) {
        cudaError_t e = cudaMalloc(&c->d_wall, wall_block_bytes(ncol, c->prec));
        if (e != cudaSuccess) {
            c->d_wall = nullptr;
            return fail(c, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,
                        std::string("lb_set_walls: ") + cudaGetErrorString(e));
        }
    }
    CK(c, cudaMemcpyAsync(wall_params(c->d_wall), params, sizeof(double) * 6 * ncol, cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, launch_wall_setup(c->prec, c->eq, c->d_wall, c->d, lattice().lc, c->stream));
    int bad = 0;
    CK(c, cudaMemcpyAsync(&bad, wall_bad_flag(c->d_wall, ncol, c->prec), sizeof bad, cudaMemcpyDeviceToHost,
                          c->stream));
    lb_status s = lb_sync(c);
    if (s != LB_OK) return s;
    if (bad) return fail(c, LB_ERR_ARG, "lb_set_walls: no equilibrium at a wall column's velocity and temperature");
    c->walls = 1;
    return LB_OK;
}

static bool wall_checks(lb_ctx* c) {
    if (c->eq == 3) {
        fail(c, LB_ERR_ARG, "lb_set_walls: walls are not combined with the entropic path length");
        return false;
    }
    if (c->d.nz < 4) {
        fail(c, LB_ERR_ARG, "lb_set_walls: walls need nz >= 4");
        return false;
    }
    return true;
}

lb_status lb_set_stochastic_rounding(lb_ctx* c, int enable, uint64_t seed) {
    if (!c) return LB_ERR_ARG;
    if (!enable) {
        c->sr = 0;
        return LB_OK;
    }
    if (c->prec != kBF16) return fail(c, LB_ERR_ARG, "lb_set_stochastic_rounding: needs BF16 storage");
    if (c->eq != 1)
        return fail(c, LB_ERR_ARG, "lb_set_stochastic_rounding: needs the series equilibrium with the projection");
    if (c->walls || c->nonideal)
        return fail(c, LB_ERR_STATE, "lb_set_stochastic_rounding: not combined with walls or the nonideal mode");
    c->sr = 1;
    c->sr_seed = seed;
    c->sr_t = 0;
    return LB_OK;
}

lb_status lb_set_walls(lb_ctx* c, int enable, const double bottom[4], const double top[4]) {
    if (!c) return LB_ERR_ARG;
    if (!enable) {
        c->walls = 0;
        return LB_OK;
    }
    if (!bottom || !top) return fail(c, LB_ERR_ARG, "lb_set_walls: null wall");
    if (c->sr) return fail(c, LB_ERR_STATE, "lb_set_walls: not combined with stochastic rounding");
    if (c->nonideal) return fail(c, LB_ERR_STATE, "lb_set_walls: not combined with the nonideal mode");
    if (!wall_checks(c)) return LB_ERR_ARG;
    if (bottom[2] != 0.0 || top[2] != 0.0) return fail(c, LB_ERR_ARG, "lb_set_walls: a wall cannot move along z");
    for (const double* w : {bottom, top})
        if (!(w[3] > 0.0) || !isfinite(w[0]) || !isfinite(w[1]) || !isfinite(w[3]))
            return fail(c, LB_ERR_ARG, "lb_set_walls: wall velocity must be finite and theta > 0");
    const int64_t ncol = (int64_t)c->d.nx * c->d.ny;
    std::vector<double> p((size_t)(6 * ncol));
    for (int side = 0; side < 2; ++side) {
        const double* w = side ? top : bottom;
        for (int k = 0; k < 3; ++k)
            std::fill(p.begin() + (side * 3 + k) * ncol, p.begin() + (side * 3 + k + 1) * ncol, w[k == 2 ? 3 : k]);
    }
    return set_wall_columns(c, p.data());
}

lb_status lb_set_wall_columns(lb_ctx* c, const double* bottom, const double* top) {
    if (!c) return LB_ERR_ARG;
    if (!bottom || !top) return fail(c, LB_ERR_ARG, "lb_set_wall_columns: null wall");
    if (!wall_checks(c)) return LB_ERR_ARG;
    const int64_t ncol = (int64_t)c->d.nx * c->d.ny;
    std::vector<double> p((size_t)(6 * ncol));
    for (int side = 0; side < 2; ++side) {
        const double* w = side ? top : bottom;
        for (int64_t k = 0; k < 3 * ncol; ++k) {
            const double v = w[k];
            if (!isfinite(v) || (k >= 2 * ncol && !(v > 0.0)))
                return fail(c, LB_ERR_ARG, "lb_set_wall_columns: wall velocity must be finite and theta > 0");
            p[(size_t)(side * 3 * ncol + k)] = v;
        }
    }
    return set_wall_columns(c, p.data());
}

// Carnahan-Starling critical packing fraction: with g(p) = p Z(p), the critical point of
// p = rho theta0 Z(b rho / 4) - a rho^2 needs g'(p) = p g''(p), i.e. the root in (0.01, 0.5) of
// (1 + 4p + 4p^2 - 4p^3 + p^4)(1 - p) - p (8 + 20p - 4p^2), found by bisection.
static double cs_critical_packing() {
    auto h = [](double p) {
        return (1 + 4 * p + 4 * p * p - 4 * p * p * p + p * p * p * p) * (1 - p) - p * (8 + 20 * p - 4 * p * p);
    };
    double lo = 0.01, hi = 0.5;  // h(lo) > 0 > h(hi)
    for (int i = 0; i < 200 && hi - lo > 1e-17; ++i) {
        const double mid = 0.5 * (lo + hi);
        (h(mid) > 0 ? lo : hi) = mid;
    }
    return 0.5 * (lo + hi);
}

lb_status lb_nonideal_constants(int eos, double theta_star, double rho_c, double* a, double* b) {
    if (!a || !b || !(theta_star > 0.0) || !(rho_c > 0.0) || !isfinite(theta_star) || !isfinite(rho_c))
        return LB_ERR_ARG;
    const double theta_c = lattice().theta0 / theta_star;
    switch (eos) {
        case LB_EOS_VAN_DER_WAALS:
            *b = 1.0 / (3.0 * rho_c);
            *a = 27.0 * *b * theta_c / 8.0;
            return LB_OK;
        case LB_EOS_PENG_ROBINSON:  // the constants printed with Eq. (cspreos)
            *a = 1.851427622 * theta_c / rho_c;
            *b = 0.353748714 / rho_c;
            return LB_OK;
        case LB_EOS_CARNAHAN_STARLING: {
            const double p = cs_critical_packing();
            const double g1 = (1 + 4 * p + 4 * p * p - 4 * p * p * p + p * p * p * p) / ((1 - p) * (1 - p) * (1 - p) * (1 - p));
            *b = 4.0 * p / rho_c;
            *a = 0.5 * g1 * theta_c / rho_c;
            return LB_OK;
        }
        default: return LB_ERR_ARG;
    }
}

lb_status lb_set_nonideal(lb_ctx* c, int enable, double a, double b, double kappa, double eta) {
    if (!c) return LB_ERR_ARG;
    if (!enable) {
        c->nonideal = 0;
        return LB_OK;
    }
    if (enable < LB_EOS_VAN_DER_WAALS || enable > LB_EOS_CARNAHAN_STARLING)
        return fail(c, LB_ERR_ARG, "lb_set_nonideal: unknown equation of state");
    if (!(a >= 0.0) || !(b > 0.0) || !(kappa >= 0.0) || !(eta >= 0.0 && eta <= 1.0) || !isfinite(a) ||
        !isfinite(b) || !isfinite(kappa))
        return fail(c, LB_ERR_ARG, "lb_set_nonideal: need a >= 0, b > 0, kappa >= 0, 0 <= eta <= 1");
    if (c->eq != 1)
        return fail(c, LB_ERR_ARG, "lb_set_nonideal: the nonideal mode uses the projected series equilibrium");
    if (c->walls) return fail(c, LB_ERR_STATE, "lb_set_nonideal: not combined with walls");
    if (c->sr) return fail(c, LB_ERR_STATE, "lb_set_nonideal: not combined with stochastic rounding");
    if (2 * c->d.plane >= ((int64_t)1 << 32))
        return fail(c, LB_ERR_ARG, "lb_set_nonideal: the grid must have fewer than 2^31 cells");
    CK(c, cudaSetDevice(c->device));
    if (!c->d_ni) {
        cudaError_t e = cudaMalloc(&c->d_ni, sizeof(double) * nonideal_doubles(c->d, c->prec));
        if (e != cudaSuccess) {
            c->d_ni = nullptr;
            return fail(c, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,
                        std::string("lb_set_nonideal: ") + cudaGetErrorString(e));
        }
    }
    c->ni_eos[0] = a;
    c->ni_eos[1] = b;
    c->ni_eos[2] = kappa;
    c->ni_eos[3] = eta;
    c->nonideal = enable;
    return LB_OK;
}

lb_status lb_wall_density(lb_ctx* c, double* rho_w) {
    if (!c || !rho_w) return LB_ERR_ARG;
    if (!c->walls) return fail(c, LB_ERR_STATE, "lb_wall_density: no walls set");
    CK(c, cudaSetDevice(c->device));
    const int64_t ncol = (int64_t)c->d.nx * c->d.ny;
    CK(c, cudaMemcpyAsync(rho_w, wall_rho(c->d_wall, ncol), sizeof(double) * 2 * ncol, cudaMemcpyDeviceToHost,
                          c->stream));
    return lb_sync(c);
}

const char* lb_last_error(const lb_ctx* c) { return c ? c->msg.c_str() : g_init_msg.c_str(); }

}  // extern "C"
