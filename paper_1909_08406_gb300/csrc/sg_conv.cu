// Surrogate kernels: periodic 3x3x3 convolution as an implicit GEMM on the
// BF16 tensor cores -- tcgen05 with the accumulator in tensor memory (the
// default), or warp-level mma.sync m16n8k16 -- with FP32 accumulation, its
// weight gradient, and the small element-wise / reduction kernels of training
// and rollout.  C ABI in include/gblb_surrogate.h.
//
// Rows are 64 voxels, periodic as a whole or (sg_shape.xper < 64) as 64 / xper
// independent segments: the d-layout of a dilated convolution (k_relabel), in
// which x + d of the volume is the next voxel of the segment.  Every kernel
// takes x +- 1 inside the segment (xseg).
//
// mma.sync forward tile: one CTA owns RT = 4 consecutive rows (64 voxels each) of one
// z-plane of one batch item: M = 256 voxels, N = cout, K = 27 * cin.  The
// CTA stages the periodic halo (3 planes x 6 rows x 66 voxels x cin) and all
// weights in shared memory with 16-byte row padding (conflict-free ldmatrix);
// each of the 16 warps computes 16 voxels x cout.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "gblb_surrogate.h"

namespace sg {

typedef __nv_bfloat16 bf16;

constexpr int kW = 64;             // voxels per row (nx)
constexpr int kRT = 4;             // rows per forward tile
constexpr int kHR = kRT + 2;       // halo rows
constexpr int kHX = kW + 2;        // halo voxels per row
constexpr int kFwdWarps = kRT * 4;  // 16 voxels per warp
constexpr int kFwdThreads = kFwdWarps * 32;

template <int CIN>
struct HaloCfg {
    static constexpr int STRIDE = CIN * 2 + 16;  // bytes per halo voxel
    static constexpr int BYTES = 3 * kHR * kHX * STRIDE;
};
template <int CIN, int COUT>
struct WCfg {
    static constexpr int STRIDE = 27 * CIN * 2 + 16;  // bytes per output channel row
    static constexpr int BYTES = COUT * STRIDE;
};

struct Epi {
    int act;
    int res_in;
    const void* add;
    int add_f32;
    float* z_out;
    int y_f32;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
// D = A * B + D, A 16x16 (row-major) BF16, B 16x8 (column-major) BF16, D 16x8 FP32
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// f(std::integral_constant<int, I>{}) for I = 0 .. N-1, unrolled at compile time
template <int... Is, class F>
__device__ __forceinline__ void sg_static_for_impl(std::integer_sequence<int, Is...>, F&& f) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    sg_static_for_impl(std::make_integer_sequence<int, N>{}, f);
}

// GELU with the Gaussian CDF, g(z) = z Phi(z), and its derivative Phi(z) + z phi(z).
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// x + dx inside the periodic segment of length L (a power of two dividing kW) that holds voxel x
// of a row: L = kW is the periodic row; L < kW splits the row into kW / L independent periodic
// segments (the layout of a dilated convolution, sg_relabel).
__device__ __forceinline__ int xseg(int x, int dx, int L) { return (x & ~(L - 1)) | ((x + dx) & (L - 1)); }

template <int CIN, int COUT>
__global__ void __launch_bounds__(kFwdThreads, 1) k_conv_fwd(sg_shape s, const bf16* __restrict__ x,
                                                              const bf16* __restrict__ w,
                                                              const float* __restrict__ bias, Epi epi, void* y) {
    using H = HaloCfg<CIN>;
    using WC = WCfg<CIN, COUT>;
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned char* halo = sm;
    unsigned char* wsm = sm + H::BYTES;
    const int tid = threadIdx.x;
    int64_t t = blockIdx.x;
    const int tiles_y = s.ny / kRT;
    const int yt = (int)(t % tiles_y);
    t /= tiles_y;
    const int z = (int)(t % s.nz);
    const int b = (int)(t / s.nz);
    const int y0 = yt * kRT;

    constexpr int CH = CIN / 8;  // 16-byte chunks per voxel
    for (int i = tid; i < 3 * kHR * kHX * CH; i += kFwdThreads) {
        const int c = i % CH;
        const int v = i / CH;
        const int xh = v % kHX, r = v / kHX;
        const int yh = r % kHR, zh = r / kHR;
        const int zz = wrapi(z + zh - 1, s.nz), yy = wrapi(y0 + yh - 1, s.ny), xx = wrapi(xh - 1, kW);
        const int64_t g = ((((int64_t)b * s.nz + zz) * s.ny + yy) * kW + xx) * CIN + c * 8;
        *reinterpret_cast<uint4*>(halo + (size_t)v * H::STRIDE + c * 16) = *reinterpret_cast<const uint4*>(x + g);
    }
    constexpr int WCH = 27 * CIN / 8;
    for (int i = tid; i < COUT * WCH; i += kFwdThreads) {
        const int co = i / WCH, c = i % WCH;
        *reinterpret_cast<uint4*>(wsm + co * WC::STRIDE + c * 16) =
            *reinterpret_cast<const uint4*>(w + (size_t)co * 27 * CIN + c * 8);
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int yl = warp >> 2, x0 = (warp & 3) * 16;
    float acc[COUT / 8][4];
#pragma unroll
    for (int i = 0; i < COUT / 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    const uint32_t hs = smem_u32(halo), ws = smem_u32(wsm);
    const int ar = lane & 15, akc = lane >> 4;
    const int bn = (lane & 7) + 8 * (lane >> 4), bkc = (lane >> 3) & 1;
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const int hrow = ((dz + 1) * kHR + (yl + 1 + dy)) * kHX + (xseg(x0 + ar, dx, s.xper) + 1);
        const uint32_t a0 = hs + hrow * H::STRIDE + akc * 16;
#pragma unroll
        for (int kb = 0; kb < CIN / 16; ++kb) {
            uint32_t a[4];
            ldsm_x4(a, a0 + kb * 32);
#pragma unroll
            for (int np = 0; np < COUT / 16; ++np) {
                uint32_t bb[4];
                ldsm_x4(bb, ws + (np * 16 + bn) * WC::STRIDE + (tap * CIN + kb * 16 + bkc * 8) * 2);
                mma_bf16(acc[2 * np], a, bb[0], bb[1]);
                mma_bf16(acc[2 * np + 1], a, bb[2], bb[3]);
            }
        }
    }

    // epilogue: lane holds (voxel g, channels 2t, 2t+1) and (voxel g + 8, same channels) per n-tile
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int nt = 0; nt < COUT / 8; ++nt) {
        const int co = nt * 8 + 2 * t4;
        const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xx = x0 + g + 8 * h;
            const int64_t v = (((int64_t)b * s.nz + z) * s.ny + (y0 + yl)) * kW + xx;
            float z0 = acc[nt][2 * h] + b0, z1 = acc[nt][2 * h + 1] + b1;
            if (epi.z_out) *reinterpret_cast<float2*>(epi.z_out + v * COUT + co) = make_float2(z0, z1);
            float o0 = epi.act == SG_ACT_GELU ? gelu(z0) : z0;
            float o1 = epi.act == SG_ACT_GELU ? gelu(z1) : z1;
            if (epi.res_in && CIN == COUT) {
                const int hc = (1 * kHR + (yl + 1)) * kHX + (xx + 1);
                const __nv_bfloat162 r = *reinterpret_cast<const __nv_bfloat162*>(halo + hc * H::STRIDE + co * 2);
                o0 += __bfloat162float(r.x);
                o1 += __bfloat162float(r.y);
            }
            if (epi.add) {
                if (epi.add_f32) {
                    const float2 r = *reinterpret_cast<const float2*>(static_cast<const float*>(epi.add) + v * COUT + co);
                    o0 += r.x;
                    o1 += r.y;
                } else {
                    const __nv_bfloat162 r =
                        *reinterpret_cast<const __nv_bfloat162*>(static_cast<const bf16*>(epi.add) + v * COUT + co);
                    o0 += __bfloat162float(r.x);
                    o1 += __bfloat162float(r.y);
                }
            }
            if (epi.y_f32)
                *reinterpret_cast<float2*>(static_cast<float*>(y) + v * COUT + co) = make_float2(o0, o1);
            else
                *reinterpret_cast<__nv_bfloat162*>(static_cast<bf16*>(y) + v * COUT + co) = __floats2bfloat162_rn(o0, o1);
        }
    }
}

// Weight gradient, split over (tap, voxel partition): CTA (tap, p) accumulates
// dw[co][tap][ci] over its voxel range in 128-voxel chunks (two rows); warp w
// takes voxels 16w..16w+15 of each chunk as the K dimension of
// D[co][ci] += dz^T[co][v] x[v + d(tap)][ci].  The 8 warps' partial sums are
// added in shared memory in a fixed order and written to partials[p][tap].
constexpr int kWgThreads = 256;
constexpr int kChunk = 128;

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgThreads) k_conv_wgrad(sg_shape s, const bf16* __restrict__ x,
                                                           const bf16* __restrict__ dz, float* __restrict__ partials,
                                                           int parts) {
    constexpr int ZS = COUT * 2 + 16, XS = CIN * 2 + 16;
    constexpr int STAGE = kChunk * (ZS + XS), RED = 8 * COUT * CIN * 4;
    // the staging tiles and, after the last chunk, the per-warp partial sums share one buffer
    __shared__ __align__(16) unsigned char buf[STAGE > RED ? STAGE : RED];
    unsigned char* zs = buf;
    unsigned char* xs = buf + kChunk * ZS;
    float (*red)[COUT * CIN] = reinterpret_cast<float (*)[COUT * CIN]>(buf);
    const int tap = blockIdx.x, p = blockIdx.y;
    const int ddz = tap / 9 - 1, ddy = (tap / 3) % 3 - 1, ddx = tap % 3 - 1;
    const int64_t voxels = (int64_t)s.batch * s.nz * s.ny * kW;
    const int64_t nchunks = voxels / kChunk;
    const int64_t c0 = nchunks * p / parts, c1 = nchunks * (p + 1) / parts;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float acc[COUT / 16][CIN / 8][4];
#pragma unroll
    for (int i = 0; i < COUT / 16; ++i)
#pragma unroll
        for (int j = 0; j < CIN / 8; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
    const uint32_t zsa = smem_u32(zs), xsa = smem_u32(xs);
    const int jm = lane >> 3, rr = lane & 7;
    for (int64_t ch = c0; ch < c1; ++ch) {
        const int64_t v0 = ch * kChunk;
        for (int i = tid; i < kChunk * (COUT / 8); i += kWgThreads) {
            const int v = i / (COUT / 8), c = i % (COUT / 8);
            *reinterpret_cast<uint4*>(zs + v * ZS + c * 16) =
                *reinterpret_cast<const uint4*>(dz + (v0 + v) * COUT + c * 8);
        }
        for (int i = tid; i < kChunk * (CIN / 8); i += kWgThreads) {
            const int v = i / (CIN / 8), c = i % (CIN / 8);
            int64_t q = v0 + v;
            const int xx = (int)(q % kW);
            q /= kW;
            const int yy = (int)(q % s.ny);
            q /= s.ny;
            const int zz = (int)(q % s.nz);
            const int bb = (int)(q / s.nz);
            const int64_t src = ((((int64_t)bb * s.nz + wrapi(zz + ddz, s.nz)) * s.ny + wrapi(yy + ddy, s.ny)) * kW +
                                 xseg(xx, ddx, s.xper)) * CIN + c * 8;
            *reinterpret_cast<uint4*>(xs + v * XS + c * 16) = *reinterpret_cast<const uint4*>(x + src);
        }
        __syncthreads();
#pragma unroll
        for (int mt = 0; mt < COUT / 16; ++mt) {
            // A = dz^T: matrix j = (co 8*(j&1).., voxels 8*(j>>1)..), rows stored by voxel -> transposed load
            uint32_t a[4];
            ldsm_x4_t(a, zsa + (16 * warp + rr + 8 * (jm >> 1)) * ZS + (16 * mt + 8 * (jm & 1)) * 2);
#pragma unroll
            for (int nt = 0; nt < CIN / 8; nt += 2) {
                // B = x: matrix j = (voxels 8*(j&1).., ci 8*(nt + (j>>1))..), rows stored by voxel -> transposed load
                uint32_t bb[4];
                ldsm_x4_t(bb, xsa + (16 * warp + rr + 8 * (jm & 1)) * XS + (8 * (nt + (jm >> 1))) * 2);
                mma_bf16(acc[mt][nt], a, bb[0], bb[1]);
                mma_bf16(acc[mt][nt + 1], a, bb[2], bb[3]);
            }
        }
        __syncthreads();
    }
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mt = 0; mt < COUT / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < CIN / 8; ++nt) {
            const int co = 16 * mt + g, ci = 8 * nt + 2 * t4;
            red[warp][co * CIN + ci] = acc[mt][nt][0];
            red[warp][co * CIN + ci + 1] = acc[mt][nt][1];
            red[warp][(co + 8) * CIN + ci] = acc[mt][nt][2];
            red[warp][(co + 8) * CIN + ci + 1] = acc[mt][nt][3];
        }
    __syncthreads();
    for (int e = tid; e < COUT * CIN; e += kWgThreads) {
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) sum += red[k][e];
        partials[((int64_t)p * 27 + tap) * COUT * CIN + e] = sum;
    }
}

// dw[co][tap][ci] = sum_p partials[p][tap][co][ci] (deterministic).  A block takes 32 consecutive
// partial entries (one per lane, coalesced); warp w adds the parts of the w-th of 8 equal ranges
// in order, then the 8 range sums are added in the order w = 0 .. 7.
__global__ void __launch_bounds__(256) k_wgrad_reduce(int cin, int cout, int parts, const float* __restrict__ partials,
                                                      float* __restrict__ dw) {
    __shared__ float sh[8][32];
    const int n = 27 * cin * cout;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int off = (int)blockIdx.x * 32 + lane;  // tap * cout * cin + co * cin + ci
    float sum = 0.f;
    if (off < n) {
        const int p0 = parts * w / 8, p1 = parts * (w + 1) / 8;
        const float* p = partials + off;
#pragma unroll 4
        for (int k = p0; k < p1; ++k) sum += p[(int64_t)k * n];
    }
    sh[w][lane] = sum;
    __syncthreads();
    if (w == 0 && off < n) {
        float t = sh[0][lane];
#pragma unroll
        for (int k = 1; k < 8; ++k) t += sh[k][lane];
        const int ci = off % cin, co = (off / cin) % cout, tap = off / (cin * cout);
        dw[((int64_t)co * 27 + tap) * cin + ci] = t;
    }
}

constexpr int kBiasBlocks = 512;  // blocks of the bias-gradient partial sums

// Partial sums of db[co] = sum_v dz[v][co] over a contiguous range of voxels per block: thread t
// reads 16-byte chunks t, t + 256, ... of the range (8 channels each; with cout / 8 chunks per
// voxel its channel group is t % (cout / 8)), then a fixed tree over the threads of one group.
__global__ void __launch_bounds__(256) k_bias_partials(int64_t voxels, int cout, const bf16* __restrict__ dz,
                                                       float* __restrict__ partial) {
    __shared__ float sh[256][8];
    const int cg = cout / 8;
    const int64_t v0 = voxels * blockIdx.x / gridDim.x, v1 = voxels * (blockIdx.x + 1) / gridDim.x;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint4* src = reinterpret_cast<const uint4*>(dz);
    for (int64_t i = v0 * cg + threadIdx.x; i < v1 * cg; i += 256) {
        const uint4 raw = src[i];
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[2 * k] += __bfloat162float(h[k].x);
            acc[2 * k + 1] += __bfloat162float(h[k].y);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    // threads of channel group g: g, g + cg, ...; halve that set in a fixed order
    for (int w = 128; w >= cg; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + w][k];
        __syncthreads();
    }
    if ((int)threadIdx.x < cg)
#pragma unroll
        for (int k = 0; k < 8; ++k) partial[(int64_t)blockIdx.x * cout + 8 * threadIdx.x + k] = sh[threadIdx.x][k];
}

// db[co] = sum over blocks of the partials, one warp per channel, fixed order: lane l adds the
// partials l, l + 32, ... (all loads issued before the additions), then a shuffle tree.
__global__ void k_bias_finish(int blocks, int cout, const float* __restrict__ partial, float* __restrict__ db) {
    const int co = (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (co >= cout) return;
    constexpr int kMaxPer = kBiasBlocks / 32;
    float v[kMaxPer];
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
        const int b = lane + 32 * j;
        v[j] = b < blocks ? partial[(int64_t)b * cout + co] : 0.f;
    }
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) sum += v[j];
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, w);
    if (lane == 0) db[co] = sum;
}

__global__ void k_act_bwd(int64_t n, int act, const float* __restrict__ dy, const float* __restrict__ z,
                          bf16* __restrict__ dz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = act == SG_ACT_GELU ? dy[i] * gelu_grad(z[i]) : dy[i];
    dz[i] = __float2bfloat16_rn(g);
}

__global__ void k_transpose_w(int cin, int cout, const bf16* __restrict__ w, bf16* __restrict__ wt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27 * cin * cout) return;
    // wt[ci][tap][co] = w[co][26 - tap][ci]
    const int co = e % cout, tap = (e / cout) % 27, ci = e / (27 * cout);
    wt[e] = w[((int64_t)co * 27 + (26 - tap)) * cin + ci];
}

constexpr int kRedBlocks = 256;

// Sum of squared differences / squares, block partials in fixed order.
__global__ void k_mse(int64_t voxels, int c, int nch, const bf16* __restrict__ pred, const bf16* __restrict__ target,
                      float* __restrict__ dpred, float* __restrict__ partial) {
    __shared__ double sh[256];
    double sum = 0.0;
    const float scale = 2.f / (float)((double)voxels * nch);
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < voxels * c; i += (int64_t)gridDim.x * 256) {
        const int ch = (int)(i % c);
        float d = 0.f;
        if (ch < nch) d = __bfloat162float(pred[i]) - __bfloat162float(target[i]);
        dpred[i] = scale * d;
        sum += (double)d * d;
    }
    sh[threadIdx.x] = sum;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = (float)sh[0];
}

__global__ void k_finish_mse(int nblocks, double denom, const float* __restrict__ partial, float* __restrict__ loss) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < nblocks; ++i) s += partial[i];
    *loss = (float)(s / denom);
}

// per batch item: sums of (a-b)^2 and b^2 over the first nch channels
__global__ void k_rel_l2(int64_t per_item, int c, int nch, const bf16* __restrict__ a, const bf16* __restrict__ b,
                         double* __restrict__ partial) {
    __shared__ double sd[256], sb[256];
    const int item = blockIdx.y;
    double d2 = 0.0, b2 = 0.0;
    const int64_t base = (int64_t)item * per_item * c;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < per_item * c; i += (int64_t)gridDim.x * 256) {
        if ((int)(i % c) >= nch) continue;
        const double av = __bfloat162float(a[base + i]), bv = __bfloat162float(b[base + i]);
        d2 += (av - bv) * (av - bv);
        b2 += bv * bv;
    }
    sd[threadIdx.x] = d2;
    sb[threadIdx.x] = b2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sd[threadIdx.x] += sd[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[((int64_t)item * gridDim.x + blockIdx.x) * 2] = sd[0];
        partial[((int64_t)item * gridDim.x + blockIdx.x) * 2 + 1] = sb[0];
    }
}

__global__ void k_finish_rel_l2(int items, int nblocks, const double* __restrict__ partial, float* __restrict__ out) {
    const int item = threadIdx.x;
    if (item >= items) return;
    double d = 0.0, b = 0.0;
    for (int i = 0; i < nblocks; ++i) {
        d += partial[((int64_t)item * nblocks + i) * 2];
        b += partial[((int64_t)item * nblocks + i) * 2 + 1];
    }
    out[item] = (float)(b > 0 ? sqrt(d / b) : sqrt(d));
}

__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ p16, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (p16) p16[i] = __float2bfloat16_rn(pi);
}

// Relabelling of a volume (nz x ny x 64 voxels per item, 2^lc 16-byte chunks per voxel) from its
// df-layout to its dt-layout (df = 2^lf, dt = 2^lt).  Voxel (b, z, y, x) sits in the d-layout at
//   b' = (b d + z mod d) d + y mod d,  z' = z / d,  y' = y / d,  x' = (x mod d)(64 / d) + x / d,
// a volume of d^2 times the items, of (nz / d) x (ny / d) x 64 voxels whose rows hold d periodic x
// segments; its neighbours at +-1 along x' (inside the segment), y' and z' are the volume's at +-d,
// so the convolution with taps d apart is the plain one of the d-layout (d = 1: the volume).
// One thread per 16-byte chunk of the destination, chunks of a voxel in adjacent lanes; 32-bit
// index arithmetic (fewer than 2^31 chunks, checked by the caller), grid-stride.
__global__ void k_relabel(int nchunks, int nz, int ny, int lc, int lf, int lt, const uint4* __restrict__ src,
                          uint4* __restrict__ dst) {
    const int nyt = ny >> lt, nzt = nz >> lt, nyf = ny >> lf, nzf = nz >> lf;
    const int mt = (1 << lt) - 1, mf = (1 << lf) - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nchunks; i += gridDim.x * blockDim.x) {
        const int c = i & ((1 << lc) - 1), t = i >> lc;
        const int xq = t & (kW - 1);
        int r = t >> 6;
        const int yq = r % nyt;
        r /= nyt;
        const int zq = r % nzt, bq = r / nzt;
        const int x = ((xq & ((kW >> lt) - 1)) << lt) | (xq >> (6 - lt));
        const int y = (yq << lt) | (bq & mt), z = (zq << lt) | ((bq >> lt) & mt), b = bq >> (2 * lt);
        const int bs = (((b << lf) | (z & mf)) << lf) | (y & mf);
        const int xs = ((x & mf) << (6 - lf)) | (x >> lf);
        const int64_t sv = (((int64_t)bs * nzf + (z >> lf)) * nyf + (y >> lf)) * kW + xs;
        dst[i] = src[(sv << lc) + c];
    }
}

// A-sub-lattice fields of one batch item -> 16 normalised channels.
__global__ void k_pack(sg_shape s, int item, const double* __restrict__ rho, const double* __restrict__ u,
                       const double* __restrict__ th, double theta0, float s0, float s1, float s2,
                       bf16* __restrict__ x) {
    const int64_t plane = (int64_t)s.nz * s.ny * s.nx;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= plane) return;
    const int64_t ustride = 2 * plane;  // u[3][2][nz][ny][nx]
    float ch[8] = {(float)((rho[q] - 1.0) / s0), (float)(u[q] / s1), (float)(u[ustride + q] / s1),
                   (float)(u[2 * ustride + q] / s1), (float)((th[q] / theta0 - 1.0) / s2), 0.f, 0.f, 0.f};
    bf16* out = x + ((int64_t)item * plane + q) * 16;
    __nv_bfloat162 pk[8];
    for (int k = 0; k < 4; ++k) pk[k] = __floats2bfloat162_rn(ch[2 * k], ch[2 * k + 1]);
    for (int k = 4; k < 8; ++k) pk[k] = __floats2bfloat162_rn(0.f, 0.f);
    uint4* o = reinterpret_cast<uint4*>(out);
    o[0] = *reinterpret_cast<uint4*>(&pk[0]);
    o[1] = *reinterpret_cast<uint4*>(&pk[4]);
}

// 16-channel prediction of one batch item -> float64 fields on both sub-lattices.
__global__ void k_unpack(sg_shape s, int item, const bf16* __restrict__ x, double theta0, float s0, float s1, float s2,
                         double* __restrict__ rho, double* __restrict__ u, double* __restrict__ th) {
    const int64_t plane = (int64_t)s.nz * s.ny * s.nx;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * plane) return;
    const int sub = q >= plane;
    const int64_t cell = q - sub * plane;
    const int xx = (int)(cell % s.nx), yy = (int)((cell / s.nx) % s.ny), zz = (int)(cell / ((int64_t)s.nx * s.ny));
    const bf16* base = x + (int64_t)item * plane * 16;
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int n = sub ? 8 : 1;
    for (int k = 0; k < n; ++k) {
        // B node of cell r sits at r + (1/2,1/2,1/2): its A neighbours are cells r + {0,1}^3
        const int ax = sub ? wrapi(xx + (k & 1), s.nx) : xx;
        const int ay = sub ? wrapi(yy + ((k >> 1) & 1), s.ny) : yy;
        const int az = sub ? wrapi(zz + (k >> 2), s.nz) : zz;
        const bf16* v = base + (((int64_t)az * s.ny + ay) * s.nx + ax) * 16;
        for (int c = 0; c < 5; ++c) acc[c] += __bfloat162float(v[c]);
    }
    const float inv = 1.f / (float)n;
    rho[q] = 1.0 + (double)(acc[0] * inv) * s0;
    u[q] = (double)(acc[1] * inv) * s1;
    u[2 * plane + q] = (double)(acc[2] * inv) * s1;
    u[4 * plane + q] = (double)(acc[3] * inv) * s1;
    th[q] = theta0 * (1.0 + (double)(acc[4] * inv) * s2);
}

// ---------------------------------------------------------------------------
// Helpers of the kernels on the 5th-generation tensor cores (tcgen05, tensor
// memory, TMA): shared-memory matrix descriptors, MMA issue and commit by one
// elected lane, bounded mbarrier waits and tensor-memory loads.  Descriptors
// follow the canonical layouts: no swizzle (8-row x 16-byte core matrices,
// LBO along K and SBO along M or N for a K-major operand) and the 32/64-byte
// swizzled layouts that TMA writes.
// ---------------------------------------------------------------------------
__device__ int g_sg_status;  // bit 0: a tensor-core wait ran out of time

// Shared-memory matrix descriptor (no swizzle): start address, leading (K)
// and stride (M/N) byte offsets, descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Warp-uniform issue: every lane forms the same operands (so they live in uniform registers) and
// one elected lane issues the instruction.
__device__ __forceinline__ void tc_mma_elect(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\tsetp.ne.u32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit_elect(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(bar)
        : "memory");
}

// true in exactly one lane of the (converged) warp
__device__ __forceinline__ bool elect_one() {
    uint32_t e;
    asm volatile("{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\tselp.b32 %0, 1, 0, p;\n}" : "=r"(e));
    return e != 0;
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.b32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory descriptor of a 32-byte-swizzled K-major operand: 8-row atoms
// of 256 B (SBO), layout type 6; the leading offset is unused for K = 16.
__device__ __forceinline__ uint64_t umma_desc_sw32(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46) |
           (6ull << 61);
}

__device__ __forceinline__ void tp_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tp_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tp_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tp_tma5(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                        uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// ---------------------------------------------------------------------------
// Forward convolution on tcgen05 with the three x taps side by side in N.
//
// A tile is 128 output voxels (two rows y0, y0 + 1 of one plane z).  For each
// (dz, dy) and 16-channel slice one tcgen05.mma multiplies the UNSHIFTED halo
// rows (A: 128 voxels x 16 channels, rows y0 + dy .. of plane z + dz) by the
// weights of the three taps dx = -1, 0, +1 of that (dz, dy) stacked along N
// (B: 3 cout x 16 channels).  Accumulator column block dxi then holds
//   D_dx[x'] = sum_(dz, dy, ci) W[co][dz, dy, dx][ci] X[z + dz, y + dy, x'][ci]
// at the lane of input voxel x', and the output is
//   y[x] = D_-1[x - 1] + D_0[x] + D_+1[x + 1]    (x periodic over the row),
// which the epilogue forms from its own lane, the neighbouring lanes (warp
// shuffles), and, at the two ends of each 32-lane quarter, the partner warp
// that holds the other half of the row (through shared memory).  Against the
// 27-tap form this reads each A operand once per (dz, dy) instead of three
// times, and keeps one copy of each halo plane instead of three x-shifted ones.
//
// Work: the tiles, numbered z fastest within a column (batch item, row pair),
// are split into one contiguous range per CTA.  A run of consecutive z within
// a column streams its planes z - 1 .. z_end through a ring of NSLOT plane
// slots (each plane: all channel slices, 4 rows x 64 voxels, 32-byte-swizzled
// K-major as TMA writes it), so tile k uses the slots of planes k, k + 1, k + 2.
// Warp roles:
//   warp 0     TMA producer (one box per slice and plane, one per row where the
//              rows wrap around the periodic y boundary)
//   warp 1     MMA issuer (9 x slices MMAs per tile, one elected lane)
//   warps 4-11 epilogue (two per tensor-memory lane quarter, half the output
//              channels each)
// All hand-offs are mbarriers and every wait is bounded; on expiry the kernel
// sets the status flag and each role waits, bounded, for its own asynchronous
// work before tensor memory is freed.
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
struct TcxCfg {
    static constexpr int K8 = CIN / 8;
    static constexpr int SL = CIN / 16;                  // 16-channel K slices
    static constexpr int HY = 4;                         // halo rows of a 2-row tile
    static constexpr int SLICEB = HY * kW * 32;          // one slice of one plane: 8 KB
    static constexpr int PLANE = SL * SLICEB;
    static constexpr int N = 3 * COUT;                   // dx-stacked output columns
    static constexpr int GB = K8 * N * 16;               // weights of one (dz, dy)
    static constexpr int B_BYTES = 9 * GB;
    static constexpr int NSLOT_FIT = (225 * 1024 - 1024 - B_BYTES) / PLANE;
    static constexpr int NSLOT = NSLOT_FIT < 12 ? NSLOT_FIT : 12;
    static constexpr int A_BYTES = NSLOT * PLANE;
    static constexpr int SMEM = A_BYTES + B_BYTES + 1024;
    static constexpr int THREADS = 640;                  // warps 0-1 roles, 2-3 spare, 4-19 epilogue
    static constexpr int EPI_GROUPS = 2;                 // epilogue groups, alternating tiles
    static constexpr int EPI_WARPS = 8;                  // per group
    static constexpr int EC = COUT / 2;                  // output channels per epilogue warp
    static constexpr int ACOLS = (N + 31) / 32 * 32;     // tensor-memory columns per accumulator
    static constexpr int NACC = 512 / ACOLS;
    static constexpr int TMEM_COLS = 512;
    static constexpr uint32_t IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    static_assert(COUT == 16 || COUT == 32, "cout: 16 or 32");
    static_assert(CIN % 16 == 0, "cin: multiple of 16");
    static_assert(NSLOT >= 4, "plane ring");
    static_assert(SMEM <= 232448 - 4096, "shared memory");
};

// Three blocks of N columns of a lane quarter (at ta, tb, tc), one wait for all three.
__device__ __forceinline__ void tc_ld3(uint32_t ta, uint32_t tb, uint32_t tc, float (&fa)[16], float (&fb)[16],
                                       float (&fc)[16]) {
    uint32_t a[16], b[16], c[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%49];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%50];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]),
          "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]), "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15]),
          "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7]), "=r"(c[8]), "=r"(c[9]), "=r"(c[10]), "=r"(c[11]), "=r"(c[12]), "=r"(c[13]), "=r"(c[14]), "=r"(c[15])
        : "r"(ta), "r"(tb), "r"(tc));
#pragma unroll
    for (int j = 0; j < 16; ++j) fa[j] = __uint_as_float(a[j]), fb[j] = __uint_as_float(b[j]), fc[j] = __uint_as_float(c[j]);
}
__device__ __forceinline__ void tc_ld3(uint32_t ta, uint32_t tb, uint32_t tc, float (&fa)[8], float (&fb)[8],
                                       float (&fc)[8]) {
    uint32_t a[8], b[8], c[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
          "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
          "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
        : "r"(ta), "r"(tb), "r"(tc));
#pragma unroll
    for (int j = 0; j < 8; ++j) fa[j] = __uint_as_float(a[j]), fb[j] = __uint_as_float(b[j]), fc[j] = __uint_as_float(c[j]);
}

// NW 32-bit words from p (16-byte aligned), and their addition to EC values: FP32 words (NW = EC)
// or pairs of bf16 (NW = EC / 2).
template <int NW>
__device__ __forceinline__ void ld_words(const uint4* p, uint32_t (&dst)[NW]) {
#pragma unroll
    for (int h = 0; h < NW / 4; ++h) {
        const uint4 raw = __ldg(p + h);
        dst[4 * h] = raw.x, dst[4 * h + 1] = raw.y, dst[4 * h + 2] = raw.z, dst[4 * h + 3] = raw.w;
    }
}
template <int EC, int NW>
__device__ __forceinline__ void add_words(float (&o)[EC], const uint32_t (&src)[NW]) {
    if constexpr (NW == EC) {
#pragma unroll
        for (int e = 0; e < EC; ++e) o[e] += __uint_as_float(src[e]);
    } else {
#pragma unroll
        for (int e = 0; e < EC / 2; ++e) {
            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&src[e]);
            o[2 * e] += __bfloat162float(h2.x);
            o[2 * e + 1] += __bfloat162float(h2.y);
        }
    }
}

// WIDE: the values loaded ahead are FP32 (an FP32 added tensor and no residual input).
template <int CIN, int COUT, bool WIDE>
__global__ void __launch_bounds__(640, 1)
    k_conv_fwd_tcx(const __grid_constant__ CUtensorMap xrows, const __grid_constant__ CUtensorMap xrow, sg_shape s,
                   const bf16* __restrict__ x, const bf16* __restrict__ w, const float* __restrict__ bias, Epi epi,
                   void* y, long long wait_limit) {
    using C = TcxCfg<CIN, COUT>;
    constexpr int EC = C::EC;
    extern __shared__ __align__(1024) unsigned char sm_tcx[];
    // barriers: plane landed, plane slot empty [NSLOT each], accumulator full, accumulator empty
    // [NACC each], row-end exchange [2 groups x 4 warp pairs], drain
    __shared__ __align__(8) uint64_t bars[2 * C::NSLOT + 2 * C::NACC + 8 + 1];
    // row-end exchange: [group][pair][warp of the pair][use parity][0: D_-1 of lane 31, 1: D_+1 of lane 0][EC]
    __shared__ float xch[2][4][2][2][2][EC];
    __shared__ uint32_t tmem_holder;
    const uint32_t base = (smem_u32(sm_tcx) + 1023u) & ~1023u;
    unsigned char* smem = sm_tcx + (base - smem_u32(sm_tcx));
    const uint32_t a_s = base, b_s = base + C::A_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int LT = 0, EM = C::NSLOT, AF = 2 * C::NSLOT, AE = AF + C::NACC, XF = AE + C::NACC, DR = XF + 8;
    auto bar = [&](int k) { return smem_u32(&bars[k]); };

    // weights: B[g = 3 (dz+1) + (dy+1)][k8][n = 3-tap column dxi * cout + co][8 channels]
    //          <- w[co][tap = 3 g + dxi][k8 * 8 ..]
    unsigned char* Bw = smem + C::A_BYTES;
    for (int i = tid; i < 27 * C::K8 * COUT; i += C::THREADS) {
        const int co = i % COUT, r = i / COUT;
        const int k8 = r % C::K8, tap = r / C::K8;
        const int g = tap / 3, dxi = tap % 3;
        *reinterpret_cast<uint4*>(Bw + (size_t)((g * C::K8 + k8) * C::N + dxi * COUT + co) * 16) =
            *reinterpret_cast<const uint4*>(w + ((size_t)co * 27 + tap) * CIN + k8 * 8);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k <= DR; ++k) {
            const int cnt = (k >= AE && k < XF) ? C::EPI_WARPS : (k >= XF && k < DR ? 4 : 1);  // AE: one group
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(k)), "r"(cnt));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;

    // tiles t = (column (b, row pair), z), z fastest; CTA c owns [t0, t1)
    const int tiles_y = s.ny / 2;
    const int64_t ntiles = (int64_t)s.batch * tiles_y * s.nz;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    // the run of tiles that starts at t: same column, consecutive z, within [t, t1)
    struct Run {
        int b, y0, z0, len;
    };
    auto run_at = [&](int64_t t) {
        const int64_t col = t / s.nz;
        const int z0 = (int)(t - col * s.nz);
        const int64_t end = min(t1, (col + 1) * (int64_t)s.nz);
        return Run{(int)(col / tiles_y), 2 * (int)(col % tiles_y), z0, (int)(end - t)};
    };
    auto fail = [&]() { atomicOr(&g_sg_status, 1); };

    if (warp == 0) {
        // ---- TMA producer: plane loads in order (run, plane); warp-uniform loop ----
        uint32_t q = 0;  // plane-load sequence number
        bool ok = true;
        for (int64_t t = t0; t < t1 && ok;) {
            const Run R = run_at(t);
            const bool y_inside = R.y0 >= 1 && R.y0 + 2 < s.ny;
            for (int p = 0; p < R.len + 2; ++p, ++q) {
                const int slot = (int)(q % C::NSLOT);
                const uint32_t use = q / C::NSLOT;
                if (!__all_sync(0xffffffffu, tc_wait(bar(EM + slot), (use & 1) ^ 1, wait_limit))) {
                    if (lane == 0) fail();
                    ok = false;
                    break;
                }
                const int zz = wrapi(R.z0 - 1 + p, s.nz);
                if (lane == 0) tp_expect_tx(bar(LT + slot), C::PLANE);
                __syncwarp();
                const uint32_t dst = a_s + (uint32_t)(slot * C::PLANE);
                if (y_inside) {
                    if (lane < C::SL)
                        tp_tma5(dst + (uint32_t)(lane * C::SLICEB), &xrows, 16 * lane, 0, R.y0 - 1, zz, R.b,
                                bar(LT + slot));
                } else if (lane < C::SL * C::HY) {
                    const int j = lane / C::HY, r = lane % C::HY;
                    tp_tma5(dst + (uint32_t)(j * C::SLICEB + r * kW * 32), &xrow, 16 * j, 0, wrapi(R.y0 + r - 1, s.ny),
                            zz, R.b, bar(LT + slot));
                }
                __syncwarp();
            }
            t += R.len;
        }
        // wait for the last use of every slot that was loaded (sequence numbers q - 1 down)
        for (uint32_t k = 0; k < (uint32_t)C::NSLOT && k < q; ++k) {
            const uint32_t sq = q - 1 - k;
            if (!__all_sync(0xffffffffu, tc_wait(bar(LT + (int)(sq % C::NSLOT)), (sq / C::NSLOT) & 1, wait_limit)) &&
                lane == 0)
                fail();
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        uint32_t q = 0;   // sequence number of the first plane of the current run
        uint32_t tt = 0;  // tile ordinal of this CTA (accumulator ring)
        bool ok = true;
        for (int64_t t = t0; t < t1 && ok;) {
            const Run R = run_at(t);
            for (int k = 0; k < R.len && ok; ++k, ++tt) {
                for (int p = (k == 0 ? 0 : k + 2); p <= k + 2; ++p) {
                    const uint32_t qq = q + p;
                    if (!__all_sync(0xffffffffu, tc_wait(bar(LT + (int)(qq % C::NSLOT)), (qq / C::NSLOT) & 1,
                                                         wait_limit))) {
                        if (lane == 0) fail();
                        ok = false;
                        break;
                    }
                }
                if (!ok) break;
                const int acc = (int)(tt % C::NACC);
                const uint32_t au = tt / C::NACC;
                if (!__all_sync(0xffffffffu, tc_wait(bar(AE + acc), (au & 1) ^ 1, wait_limit))) {
                    if (lane == 0) fail();
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d_tmem = tmem + (uint32_t)(acc * C::ACOLS);
                const uint64_t a_pl[3] = {umma_desc_sw32(a_s + ((q + k) % C::NSLOT) * C::PLANE),
                                          umma_desc_sw32(a_s + ((q + k + 1) % C::NSLOT) * C::PLANE),
                                          umma_desc_sw32(a_s + ((q + k + 2) % C::NSLOT) * C::PLANE)};
                const uint64_t b0 = umma_desc(b_s, C::N * 16, 128);
                static_for<C::SL>([&](auto J) {
                    static_for<9>([&](auto G) {
                        constexpr int dz = G / 3, dy = G % 3;  // each + 1
                        constexpr uint64_t aoff = (uint64_t)((J * C::SLICEB + dy * kW * 32) >> 4);
                        constexpr uint64_t boff = (uint64_t)(((G * C::K8 + 2 * J) * C::N * 16) >> 4);
                        tc_mma_elect(d_tmem, a_pl[dz] + aoff, b0 + boff, C::IDESC, (J == 0 && G == 0) ? 0u : 1u);
                    });
                });
                // plane k is not used by later tiles of the run; the last tile frees all three
                tc_commit_elect(bar(EM + (int)((q + k) % C::NSLOT)));
                if (k == R.len - 1) {
                    tc_commit_elect(bar(EM + (int)((q + k + 1) % C::NSLOT)));
                    tc_commit_elect(bar(EM + (int)((q + k + 2) % C::NSLOT)));
                }
                tc_commit_elect(bar(AF + acc));
            }
            q += R.len + 2;
            t += R.len;
        }
        // every MMA this warp issued has completed before tensor memory can be freed
        tc_commit_elect(bar(DR));
        if (!__all_sync(0xffffffffu, tc_wait(bar(DR), 0, wait_limit)) && lane == 0) fail();
    } else if (warp >= 4) {
        // ---- epilogue: group grp takes the tiles tt = grp, grp + 2, ...; a warp reads lanes
        // 32 (warp % 4) .. + 31 and output channels half * EC .. + EC ----
        const int grp = (warp - 4) >> 3, quarter = warp & 3, half = ((warp - 4) >> 2) & 1;
        const int c_lo = half * EC;
        const int m = 32 * quarter + lane;
        const int yl = m >> 6, xx = m & 63;
        const int pair = half * 2 + yl, pw = quarter & 1;  // the two quarters of a row form a pair
        const bool seg = s.xper < kW;  // rows of independent periodic segments (within a quarter)
        // the residual input (or, without one, the added values) of a tile is loaded one tile of
        // this group ahead: EC bf16 values in EC / 2 words, or EC FP32 values in EC words
        const bool res = epi.res_in && CIN == COUT;
        const bool pre_add = !res && epi.add;
        const bool bias4 = bias && ((uintptr_t)bias & 15) == 0;
        constexpr int XW = WIDE ? EC : EC / 2;  // 32-bit words loaded ahead
        uint32_t nxt[XW];
        auto voxel_of = [&](const Run& R, int k) {
            return (((int64_t)R.b * s.nz + (R.z0 + k)) * s.ny + (R.y0 + yl)) * kW + xx;
        };
        // EC bf16 values (EC / 2 words) or EC FP32 values (EC words) of voxel v: the residual input
        // or the added tensor
        auto extra_ptr = [&](int64_t v, bool is_res, bool f32) {
            return is_res ? reinterpret_cast<const uint4*>(x + v * CIN + c_lo)
                          : (f32 ? reinterpret_cast<const uint4*>(static_cast<const float*>(epi.add) + v * COUT + c_lo)
                                 : reinterpret_cast<const uint4*>(static_cast<const bf16*>(epi.add) + v * COUT + c_lo));
        };
        // the tiles of this group in order
        int64_t t = t0;
        Run R = run_at(t);
        int k = 0;
        auto advance = [&](int steps) {  // move (t, R, k) forward by `steps` tiles
            for (int i = 0; i < steps && t < t1; ++i) {
                ++t;
                if (++k == R.len && t < t1) {
                    R = run_at(t);
                    k = 0;
                }
            }
        };
        advance(grp);
        if (t < t1 && (res || pre_add)) ld_words(extra_ptr(voxel_of(R, k), res, WIDE), nxt);
        uint32_t tt = (uint32_t)grp, use = 0;
        bool ok = true;
        while (t < t1 && ok) {
            const int64_t v = voxel_of(R, k);
            uint32_t cur[XW];
#pragma unroll
            for (int i = 0; i < XW; ++i) cur[i] = nxt[i];
            advance(C::EPI_GROUPS);
            if (t < t1 && (res || pre_add)) ld_words(extra_ptr(voxel_of(R, k), res, WIDE), nxt);

            const int acc = (int)(tt % C::NACC);
            const uint32_t au = tt / C::NACC;
            if (!__all_sync(0xffffffffu, tc_wait(bar(AF + acc), au & 1, wait_limit))) {
                if (lane == 0) fail();
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // z[x] = D_-1[x - 1] + D_0[x] + D_+1[x + 1]; lane 0's left and lane 31's right term
            // come from the partner warp, which holds the other half of the row
            const int par = (int)(use & 1);
            const int xb = XF + 4 * grp + pair;
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(acc * C::ACOLS + c_lo);
            float zc[EC];
            {
                float dm[EC], dp[EC];
                tc_ld3(taddr, taddr + COUT, taddr + 2 * COUT, dm, zc, dp);  // D_-1, D_0, D_+1
                if (lane == 31) {
#pragma unroll
                    for (int e = 0; e < EC; ++e) xch[grp][pair][pw][par][0][e] = dm[e];
                }
                if (lane == 0) {
#pragma unroll
                    for (int e = 0; e < EC; ++e) xch[grp][pair][pw][par][1][e] = dp[e];
                }
                if (seg) {
                    // x-period L <= 32: the segment lies inside this warp's 32 voxels
                    const int sl = xseg(lane, -1, s.xper), sr = xseg(lane, 1, s.xper);
#pragma unroll
                    for (int e = 0; e < EC; ++e)
                        zc[e] += __shfl_sync(0xffffffffu, dm[e], sl) + __shfl_sync(0xffffffffu, dp[e], sr);
                } else {
#pragma unroll
                    for (int e = 0; e < EC; ++e) {
                        const float l = __shfl_up_sync(0xffffffffu, dm[e], 1);
                        const float r = __shfl_down_sync(0xffffffffu, dp[e], 1);
                        zc[e] += (lane == 0 ? 0.f : l) + (lane == 31 ? 0.f : r);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) tp_arrive(bar(AE + acc));
            if (lane == 0 || lane == 31) tp_arrive(bar(xb));
            if (!__all_sync(0xffffffffu, tc_wait(bar(xb), use & 1, wait_limit))) {
                if (lane == 0) fail();
                ok = false;
                break;
            }
            if (lane == 0 && !seg) {
#pragma unroll
                for (int e = 0; e < EC; ++e) zc[e] += xch[grp][pair][pw ^ 1][par][0][e];
            }
            if (lane == 31 && !seg) {
#pragma unroll
                for (int e = 0; e < EC; ++e) zc[e] += xch[grp][pair][pw ^ 1][par][1][e];
            }
            if (bias4) {
#pragma unroll
                for (int e = 0; e < EC / 4; ++e) {
                    const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + c_lo) + e);
                    zc[4 * e] += b4.x, zc[4 * e + 1] += b4.y, zc[4 * e + 2] += b4.z, zc[4 * e + 3] += b4.w;
                }
            } else if (bias) {
#pragma unroll
                for (int e = 0; e < EC; ++e) zc[e] += __ldg(bias + c_lo + e);
            }
            if (epi.z_out) {
                float4* zo = reinterpret_cast<float4*>(epi.z_out + v * COUT + c_lo);
#pragma unroll
                for (int e = 0; e < EC / 4; ++e) zo[e] = make_float4(zc[4 * e], zc[4 * e + 1], zc[4 * e + 2], zc[4 * e + 3]);
            }
            if (epi.act == SG_ACT_GELU) {
#pragma unroll
                for (int e = 0; e < EC; ++e) zc[e] = gelu(zc[e]);
            }
            if (res || pre_add) add_words(zc, cur);
            if (res && epi.add) {  // both a residual and an added tensor: the added one read here
                if (epi.add_f32) {
                    uint32_t ex[EC];
                    ld_words(extra_ptr(v, false, true), ex);
                    add_words(zc, ex);
                } else {
                    uint32_t ex[EC / 2];
                    ld_words(extra_ptr(v, false, false), ex);
                    add_words(zc, ex);
                }
            }
            if (epi.y_f32) {
                float4* yo = reinterpret_cast<float4*>(static_cast<float*>(y) + v * COUT + c_lo);
#pragma unroll
                for (int e = 0; e < EC / 4; ++e) yo[e] = make_float4(zc[4 * e], zc[4 * e + 1], zc[4 * e + 2], zc[4 * e + 3]);
            } else {
                uint4 pk[EC / 8];
                __nv_bfloat162* pp = reinterpret_cast<__nv_bfloat162*>(pk);
#pragma unroll
                for (int e = 0; e < EC / 2; ++e) pp[e] = __floats2bfloat162_rn(zc[2 * e], zc[2 * e + 1]);
                uint4* yo = reinterpret_cast<uint4*>(static_cast<bf16*>(y) + v * COUT + c_lo);
#pragma unroll
                for (int h = 0; h < EC / 8; ++h) yo[h] = pk[h];
            }
            tt += C::EPI_GROUPS;
            ++use;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
}

// ---------------------------------------------------------------------------
// Weight gradient on tcgen05 (TMA operands, accumulators in tensor memory).
//
//   dw[co][tap][ci] = sum_v dz[v][co] x[v + d(tap)][ci],  d(tap) = (dz, dy, dx)
//
// Over one row (b, z, y) of 64 voxels, with x' = x + dx taken periodically,
//   sum_x dZ[b,z,y,x][co] X[b,z+dz,y+dy,x+dx][ci]
//     = sum_x' X[b,z+dz,y+dy,x'][ci] dZ[b,z,y,x'-dx][co],
// a GEMM with K = the 64 voxels x' of the row:
//   A[m][k] = X row (z+dz, y+dy) at voxel k,  m = (dz, dy, ci): 9 cin rows,
//   B[k][n] = dZ row (z, y) at voxel k - dx,  n = (dx, co):     N = 3 cout.
// Both operands are MN-major, i.e. channels contiguous, which is the
// activations' own [voxel][channel] layout: one TMA box writes an x row with
// all its channels (32 or 64 bytes per voxel) as one column of the 32- or
// 64-byte swizzled layout (LBO = the column's bytes between atoms along M or
// N, SBO = 8 voxels along K), so the k-th 16-voxel step of an MMA is a start
// address 16 voxels further on.  The producer issues a stage's boxes from as
// many lanes, one box each.  Rows are taken in pairs (y, y + 1): one A stage
// holds the 12 x rows (z + dz, y + dy'), dy' = -1 .. 2, at positions
// p = 3 (dy' + 1) + (dz + 1), so output row y + j reads the window of 9
// positions starting at 3 j, in the same (dy, dz) order, and the pair loads 12
// x rows instead of 18.  The 9 rows of a window are cut into M = 128 tiles of
// 128 / cin rows (the last tile padded with rows whose products are
// discarded); B holds each dZ row of the pair in three copies shifted by dx = -1, 0, +1:
// each copy is one 64-voxel box starting one voxel before or after the row
// (every box lands on a column boundary), whose out-of-range voxel the tensor
// map fills with zeros and a fixer warp then overwrites, at its swizzled place,
// with the periodic wrap voxel.  A CTA owns a contiguous range of row pairs and
// accumulates each tile's D[128][3 cout] (FP32) in tensor memory over all of
// them; the epilogue writes the CTA's partial dw, summed over CTAs in a fixed
// order by k_wgrad_reduce.
// Warp roles: warp 0 TMA producer, warp 1 MMA issuer (warp-uniform loops, one
// elected lane issues), warp 2 wrap-voxel fixer, warps 4-7 epilogue (one
// tensor-memory lane quarter each).  Every wait is bounded; on expiry the status flag is set and each
// role waits, bounded, for its own asynchronous work before tensor memory is
// freed.
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
struct WgCfg {
    static constexpr int RA = 2 * CIN;                  // bytes of one voxel's channels in A (32 or 64)
    static constexpr int RB = 2 * COUT;                 // and in B
    static constexpr int COLA = 64 * RA;                // one x row: a column (swizzle atom group) of A
    static constexpr int COLB = 64 * RB;                // one shifted dz row: a column of B
    static constexpr int PER_TILE = 128 / CIN;          // columns of A per M = 128 tile
    static constexpr int NT = (9 + PER_TILE - 1) / PER_TILE;  // tiles over the 9 (dz, dy) rows
    static constexpr int N = 3 * COUT;                  // B columns: (dx, co)
    static constexpr int NS = (N + 31) / 32 * 32;       // tensor-memory columns per tile (32-aligned)
    static constexpr int NLOAD = 12;                    // x rows loaded per row pair
    static constexpr int NPOS = 3 + PER_TILE * NT;      // positions the two windows' tiles reach
    static constexpr int A_STAGE = NPOS * COLA;         // one row pair's x rows
    static constexpr int B_STAGE = 2 * 3 * COLB;        // one row pair's shifted dZ rows
    static constexpr int SB = 3;                        // B stages
    static constexpr int SA = (220 * 1024 - SB * B_STAGE) / A_STAGE;  // A stages
    static constexpr int SMEM = SA * A_STAGE + SB * B_STAGE + 1024;
    static constexpr int TMEM_USED = NT * NS;
    static constexpr int TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 : TMEM_USED <= 128 ? 128
                                     : TMEM_USED <= 256 ? 256 : 512;
    static constexpr int THREADS = 256;
    // layout types of the shared-memory descriptors: 32- or 64-byte swizzle
    static constexpr uint64_t SWA = RA == 64 ? 4 : 6, SWB = RB == 64 ? 4 : 6;
    // D F32, A and B BF16, both MN-major (bits 15, 16), N, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                      ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    static_assert((CIN == 16 || CIN == 32) && (COUT == 16 || COUT == 32), "16 or 32 channels");
    static_assert(N % 16 == 0 && N <= 256, "N = 3 cout must be a multiple of 16, at most 256");
    static_assert(TMEM_USED <= 512, "tensor memory");
    static_assert(SMEM <= 232448, "shared memory");
    static_assert(SA >= 2, "A stages");
};

// Shared-memory descriptor of a swizzled MN-major operand: start address, LBO = stride between
// atoms along M (N), SBO = stride between groups of 8 rows along K, layout type (6: 32-byte, 4:
// 64-byte swizzle), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint64_t layout) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46) | (layout << 61);
}

// 16-byte chunk c of row v of a swizzled row of R bytes (R = 32: 32-byte swizzle, rows 4..7 of
// each 8-row group swap their halves; R = 64: 64-byte swizzle, chunk c ^ ((v >> 1) & 3))
template <int R>
__device__ __forceinline__ uint32_t swz_chunk(int v, int c) {
    return (uint32_t)(R == 64 ? (c ^ ((v >> 1) & 3)) : (c ^ ((v >> 2) & 1)));
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(256, 1)
    k_conv_wgrad_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap zmap, sg_shape s,
                    const bf16* __restrict__ dzg, float* __restrict__ partials, float* __restrict__ bias_part,
                    long long wait_limit) {
    using C = WgCfg<CIN, COUT>;
    extern __shared__ __align__(1024) unsigned char sm_wg[];
    // barriers: A full, A empty [SA]; B landed, B full, B empty [SB]; done
    __shared__ __align__(8) uint64_t bars[2 * C::SA + 3 * C::SB + 1];
    __shared__ uint32_t tmem_holder;
    const uint32_t base = (smem_u32(sm_wg) + 1023u) & ~1023u;
    const uint32_t a_s = base, b_s = base + C::SA * C::A_STAGE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int AF = 0, AE = C::SA, BL = 2 * C::SA, BF = BL + C::SB, BE = BF + C::SB, DN = BE + C::SB;
    auto bar = [&](int k) { return smem_u32(&bars[k]); };
    auto fail = [&]() { atomicOr(&g_sg_status, 1); };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        // a B stage is empty once the MMAs have read it and, with a bias gradient, the fixer has summed it
        for (int k = 0; k <= DN; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(k)),
                         "r"(k >= BE && k < BE + C::SB && bias_part ? 2 : 1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;

    // this CTA's row pairs [r0, r1) of the batch x nz x ny / 2 pairs (y, y + 1) of 64-voxel rows
    const int hy = s.ny / 2;
    const int64_t rows = (int64_t)s.batch * s.nz * hy;
    const int64_t r0 = rows * blockIdx.x / gridDim.x, r1 = rows * (blockIdx.x + 1) / gridDim.x;
    auto row_coord = [&](int64_t r, int& b, int& z, int& y) {  // y: the pair's first row
        y = 2 * (int)(r % hy);
        const int64_t q = r / hy;
        z = (int)(q % s.nz);
        b = (int)(q / s.nz);
    };

    if (warp == 0) {
        // ---- TMA producer: per row pair, the six shifted dZ copies, then the 12 x rows ----
        uint32_t qa = 0, qb = 0;  // A / B stage sequence numbers
        bool ok = true;
        for (int64_t r = r0; r < r1 && ok; ++r) {
            int b, z, y;
            row_coord(r, b, z, y);
            {
                const int st = (int)(qb % C::SB);
                const uint32_t use = qb / C::SB;
                if (!__all_sync(0xffffffffu, tc_wait(bar(BE + st), (use & 1) ^ 1, wait_limit))) {
                    if (lane == 0) fail();
                    ok = false;
                    break;
                }
                // one box per lane (a TMA issue from one lane takes ~140 cycles; the lanes issue in
                // parallel), after lane 0 has posted the stage's byte count
                if (lane == 0) tp_expect_tx(bar(BL + st), C::B_STAGE);
                __syncwarp();
                if (lane < 6) {
                    // copy dxi of row y + j holds dZ[(x' - dx) mod 64], dx = dxi - 1: a box starting at
                    // voxel -dx (dx = +1: voxel 0 out of range; dx = -1: voxel 63 out of range)
                    const int j = lane / 3, dxi = lane % 3;
                    tp_tma5(b_s + (uint32_t)(st * C::B_STAGE + (3 * j + dxi) * C::COLB), &zmap, 0, 1 - dxi, y + j, z,
                            b, bar(BL + st));
                }
                __syncwarp();
                ++qb;
            }
            {
                const int st = (int)(qa % C::SA);
                const uint32_t use = qa / C::SA;
                if (!__all_sync(0xffffffffu, tc_wait(bar(AE + st), (use & 1) ^ 1, wait_limit))) {
                    if (lane == 0) fail();
                    ok = false;
                    break;
                }
                // position p = 3 (dy' + 1) + (dz + 1) holds the x row (z + dz, y + dy'), dy' = -1 .. 2
                if (lane == 0) tp_expect_tx(bar(AF + st), (uint32_t)(C::NLOAD * C::COLA));
                __syncwarp();
                if (lane < C::NLOAD) {
                    const int dy = lane / 3 - 1, dz = lane % 3 - 1;
                    tp_tma5(a_s + (uint32_t)(st * C::A_STAGE + lane * C::COLA), &xmap, 0, 0, wrapi(y + dy, s.ny),
                            wrapi(z + dz, s.nz), b, bar(AF + st));
                }
                __syncwarp();
                ++qa;
            }
        }
        // the CTA must not exit with boxes still landing: wait for the last use of every stage
        for (uint32_t k = 0; k < (uint32_t)C::SA && k < qa; ++k) {
            const uint32_t sq = qa - 1 - k;
            if (!__all_sync(0xffffffffu, tc_wait(bar(AF + (int)(sq % C::SA)), (sq / C::SA) & 1, wait_limit)) &&
                lane == 0)
                fail();
        }
        for (uint32_t k = 0; k < (uint32_t)C::SB && k < qb; ++k) {
            const uint32_t sq = qb - 1 - k;
            if (!__all_sync(0xffffffffu, tc_wait(bar(BL + (int)(sq % C::SB)), (sq / C::SB) & 1, wait_limit)) &&
                lane == 0)
                fail();
        }
    } else if (warp == 2) {
        // ---- wrap-voxel fixer: per row pair and x segment g (length L = xper; one segment for a
        // periodic row), item (j, side, c8) writes one 16-byte chunk of a shifted copy's wrap voxel
        // of row y + j: side 0 (dx = +1, copy 2) voxel g L <- dZ[g L + L - 1]; side 1 (dx = -1,
        // copy 0) voxel g L + L - 1 <- dZ[g L], at its swizzled place.  The 4 cout/8 items of a
        // segment go to consecutive lanes, all loads issued before the stage's wait ----
        constexpr int COG = COUT / 8, PER_SEG = 4 * COG, KMAX = (PER_SEG * (kW / 8) + 31) / 32;
        const int L = s.xper, items = PER_SEG * (kW / L);
        float bsum = 0.f;
        uint32_t qb = 0;
        for (int64_t r = r0; r < r1; ++r, ++qb) {
            int b, z, y;
            row_coord(r, b, z, y);
            const int st = (int)(qb % C::SB);
            uint4 val[KMAX];
#pragma unroll
            for (int i = 0; i < KMAX; ++i) {
                const int it = lane + 32 * i, g = it / PER_SEG, rem = it % PER_SEG;
                const int j = rem / (2 * COG), side = (rem / COG) & 1, c8 = rem % COG;
                val[i] = make_uint4(0, 0, 0, 0);
                if (it < items)
                    val[i] = *reinterpret_cast<const uint4*>(
                        dzg + ((((int64_t)b * s.nz + z) * s.ny + y + j) * kW + (side ? g * L : g * L + L - 1)) * COUT +
                        8 * c8);
            }
            if (!__all_sync(0xffffffffu, tc_wait(bar(BL + st), (qb / C::SB) & 1, wait_limit))) {
                if (lane == 0) fail();
                break;
            }
#pragma unroll
            for (int i = 0; i < KMAX; ++i) {
                const int it = lane + 32 * i, g = it / PER_SEG, rem = it % PER_SEG;
                const int j = rem / (2 * COG), side = (rem / COG) & 1, c8 = rem % COG;
                const int v = side ? g * L + L - 1 : g * L;
                const uint32_t dst = b_s +
                                     (uint32_t)(st * C::B_STAGE + (3 * j + (side ? 0 : 2)) * C::COLB + v * C::RB) +
                                     16u * swz_chunk<C::RB>(v, c8);
                if (it < items)
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(val[i].x), "r"(val[i].y),
                                 "r"(val[i].z), "r"(val[i].w)
                                 : "memory");
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) tp_arrive(bar(BF + st));
            if (bias_part) {
                // bias gradient: lane co adds dZ[x][co] of the pair's unshifted copies (copy 1), x in order
                if (lane < COUT) {
#pragma unroll 1
                    for (int jj = 0; jj < 2; ++jj) {
                        const uint32_t cb = b_s + (uint32_t)(st * C::B_STAGE + (3 * jj + 1) * C::COLB);
#pragma unroll 8
                        for (int x = 0; x < kW; ++x) {
                            unsigned short hv;
                            const uint32_t a = cb + (uint32_t)(x * C::RB) + 16u * swz_chunk<C::RB>(x, lane >> 3) +
                                               2u * (uint32_t)(lane & 7);
                            asm volatile("ld.shared.u16 %0, [%1];" : "=h"(hv) : "r"(a));
                            bsum += __bfloat162float(__ushort_as_bfloat16(hv));
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) tp_arrive(bar(BE + st));
            }
        }
        if (bias_part && lane < COUT) bias_part[(int64_t)blockIdx.x * COUT + lane] = bsum;
    } else if (warp == 1) {
        // ---- MMA issuer ----
        uint32_t qa = 0, qb = 0;
        bool ok = true, first = true;
        for (int64_t r = r0; r < r1 && ok; ++r) {
            const int bst = (int)(qb % C::SB);
            if (!__all_sync(0xffffffffu, tc_wait(bar(BF + bst), (qb / C::SB) & 1, wait_limit))) {
                if (lane == 0) fail();
                ok = false;
                break;
            }
            const int st = (int)(qa % C::SA);
            if (!__all_sync(0xffffffffu, tc_wait(bar(AF + st), (qa / C::SA) & 1, wait_limit))) {
                if (lane == 0) fail();
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int j = 0; j < 2; ++j) {
                // row y + j: its three shifted dZ copies, and the window of x rows starting at position 3 j
                const uint64_t bdesc =
                    umma_desc_mn(b_s + (uint32_t)(bst * C::B_STAGE + 3 * j * C::COLB), C::COLB, 8 * C::RB, C::SWB);
                for (int t = 0; t < C::NT; ++t) {
                    const uint64_t adesc = umma_desc_mn(
                        a_s + (uint32_t)(st * C::A_STAGE + (3 * j + C::PER_TILE * t) * C::COLA), C::COLA, 8 * C::RA,
                        C::SWA);
                    const uint32_t d_tmem = tmem + (uint32_t)(t * C::NS);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)  // 16 voxels per MMA: start address + 16 rows
                        tc_mma_elect(d_tmem, adesc + (uint64_t)((16 * C::RA * kk) >> 4),
                                     bdesc + (uint64_t)((16 * C::RB * kk) >> 4), C::IDESC,
                                     (first && j == 0 && kk == 0) ? 0u : 1u);
                }
            }
            tc_commit_elect(bar(AE + st));
            tc_commit_elect(bar(BE + bst));
            ++qa;
            ++qb;
            first = false;
        }
        // every MMA this warp issued has completed before the epilogue reads or tensor memory is freed
        tc_commit_elect(bar(DN));
        if (!__all_sync(0xffffffffu, tc_wait(bar(DN), 0, wait_limit)) && lane == 0) fail();
    } else if (warp >= 4) {
        // ---- epilogue: lanes 32 q .. 32 q + 31 of each tile, all N columns ----
        const int q = warp & 3;
        const bool ok = __all_sync(0xffffffffu, tc_wait(bar(DN), 0, wait_limit));
        if (!ok) {
            if (lane == 0) fail();
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float* out = partials + (int64_t)blockIdx.x * 27 * COUT * CIN;
            const int m = 32 * q + lane;
            for (int t = 0; t < C::NT; ++t) {
                // row m of tile t: window position p = PER_TILE t + m / cin = 3 (dy + 1) + (dz + 1),
                // channel m % cin
                const int p = C::PER_TILE * t + m / CIN, ci = m % CIN;
                const bool real = p < 9;
                const int dy = p / 3 - 1, dz = p % 3 - 1;
#pragma unroll
                for (int n0 = 0; n0 < C::N; n0 += 16) {
                    float v[16];
                    tc_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(t * C::NS + n0), v);
                    if (real) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int n = n0 + j, dxi = n / COUT, co = n - dxi * COUT;
                            const int tap = (dz + 1) * 9 + (dy + 1) * 3 + dxi;
                            out[(int64_t)tap * COUT * CIN + co * CIN + ci] = v[j];
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
}

static int g_fwd_impl = SG_CONV_TCGEN05;  // forward convolution kernel (sg_set_conv_impl)

// cuTensorMapEncodeTiled from the driver, found once through the runtime (no link-time driver dependency)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

template <int CIN, int COUT>
static int launch_fwd_tcx(sg_shape s, const void* x, const void* w, const float* bias, Epi epi, void* y,
                          cudaStream_t st) {
    using C = TcxCfg<CIN, COUT>;
    static int configured = -1, grid_max = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -3;
    if (configured != dev) {
        if (cudaFuncSetAttribute(k_conv_fwd_tcx<CIN, COUT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(k_conv_fwd_tcx<CIN, COUT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::SMEM) != cudaSuccess)
            return -3;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -3;
        grid_max = sms;  // one CTA per SM (shared memory, all of tensor memory)
        configured = dev;
    }
    auto encode = tensor_map_encoder();
    if (!encode) return -3;
    // activations x[b][z][y][x][c] as a 5D tensor (c fastest); boxes of 16 channels (32 bytes, the
    // swizzle span) x 64 voxels x 4 rows or x 1 row, written 32-byte swizzled
    const cuuint64_t dims[5] = {(cuuint64_t)CIN, (cuuint64_t)kW, (cuuint64_t)s.ny, (cuuint64_t)s.nz, (cuuint64_t)s.batch};
    const cuuint64_t strides[4] = {(cuuint64_t)CIN * 2, (cuuint64_t)kW * CIN * 2, (cuuint64_t)s.ny * kW * CIN * 2,
                                   (cuuint64_t)s.nz * s.ny * kW * CIN * 2};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    alignas(64) CUtensorMap rows, row;
    const cuuint32_t box_rows[5] = {16, (cuuint32_t)kW, (cuuint32_t)C::HY, 1, 1};
    const cuuint32_t box_row[5] = {16, (cuuint32_t)kW, 1, 1, 1};
    if (encode(&rows, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dims, strides, box_rows, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        encode(&row, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dims, strides, box_row, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return -3;
    const int64_t tiles = (int64_t)s.batch * (s.ny / 2) * s.nz;
    const int grid = (int)(tiles < grid_max ? tiles : grid_max);
    const long long wait_limit = 2000000000LL;  // ~1 s of SM clock per wait
    const bool wide = !(epi.res_in && CIN == COUT) && epi.add && epi.add_f32;
    auto kern = wide ? k_conv_fwd_tcx<CIN, COUT, true> : k_conv_fwd_tcx<CIN, COUT, false>;
    kern<<<grid, C::THREADS, C::SMEM, st>>>(rows, row, s, static_cast<const bf16*>(x), static_cast<const bf16*>(w),
                                            bias, epi, y, wait_limit);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <int CIN, int COUT>
static int launch_fwd(sg_shape s, const void* x, const void* w, const float* bias, Epi epi, void* y,
                      cudaStream_t st) {
    if (g_fwd_impl == SG_CONV_TCGEN05) return launch_fwd_tcx<CIN, COUT>(s, x, w, bias, epi, y, st);
    constexpr int smem = HaloCfg<CIN>::BYTES + WCfg<CIN, COUT>::BYTES;
    static int configured = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -3;
    if (configured != dev) {
        if (cudaFuncSetAttribute(k_conv_fwd<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
            return -3;
        configured = dev;
    }
    const int64_t tiles = (int64_t)s.batch * s.nz * (s.ny / kRT);
    k_conv_fwd<CIN, COUT><<<(unsigned)tiles, kFwdThreads, smem, st>>>(
        s, static_cast<const bf16*>(x), static_cast<const bf16*>(w), bias, epi, y);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

static int parts_for(sg_shape s) {
    const int64_t chunks = (int64_t)s.batch * s.nz * s.ny * kW / kChunk;
    int p = 32;
    if (p > chunks) p = (int)chunks;
    return p < 1 ? 1 : p;
}

constexpr int kWgMaxCtas = 160;  // partial sums of the tcgen05 weight gradient: at most one per CTA

// CTAs of the tcgen05 weight gradient for this shape (one per SM, at most one per row).
static int wgrad_tc_ctas(sg_shape s) {
    static int sms = 0, dev_seen = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (dev != dev_seen) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
        dev_seen = dev;
    }
    int64_t n = sms < kWgMaxCtas ? sms : kWgMaxCtas;
    const int64_t pairs = (int64_t)s.batch * s.nz * (s.ny / 2);
    if (n > pairs) n = pairs;
    return (int)n;
}

template <int CIN, int COUT>
static int launch_wgrad_tc(sg_shape s, const void* x, const void* dz, float* partials, float* bias_part, int ctas,
                           cudaStream_t st) {
    using C = WgCfg<CIN, COUT>;
    static int configured = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -3;
    if (configured != dev) {
        if (cudaFuncSetAttribute(k_conv_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) !=
            cudaSuccess)
            return -3;
        configured = dev;
    }
    auto encode = tensor_map_encoder();
    if (!encode) return -3;
    // x[b][z][y][x][ci], dz[b][z][y][x][co] as 5D tensors (channels fastest); boxes of all channels
    // x 64 voxels of one row, 32- or 64-byte swizzled: one column of a swizzled MN-major operand
    auto enc = [&](CUtensorMap* m, const void* ptr, int ch) {
        const cuuint64_t dims[5] = {(cuuint64_t)ch, (cuuint64_t)kW, (cuuint64_t)s.ny, (cuuint64_t)s.nz,
                                    (cuuint64_t)s.batch};
        const cuuint64_t strides[4] = {(cuuint64_t)ch * 2, (cuuint64_t)kW * ch * 2, (cuuint64_t)s.ny * kW * ch * 2,
                                       (cuuint64_t)s.nz * s.ny * kW * ch * 2};
        const cuuint32_t box[5] = {(cuuint32_t)ch, (cuuint32_t)kW, 1, 1, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(ptr), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, ch == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    alignas(64) CUtensorMap xm, zm;
    if (!enc(&xm, x, CIN) || !enc(&zm, dz, COUT)) return -3;
    const long long wait_limit = 2000000000LL;  // ~1 s of SM clock per wait
    k_conv_wgrad_tc<CIN, COUT><<<ctas, C::THREADS, C::SMEM, st>>>(xm, zm, s, static_cast<const bf16*>(dz), partials,
                                                                   bias_part,
                                                                   wait_limit);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Weight-gradient partial sums either kernel may write: the mma.sync one's voxel partitions or the
// tcgen05 one's CTAs (at most one per row, at most kWgMaxCtas).
static int64_t wgrad_parts_max(sg_shape s) {
    const int64_t rows = (int64_t)s.batch * s.nz * s.ny;
    const int64_t tc = rows < kWgMaxCtas ? rows : kWgMaxCtas;
    const int64_t mma = parts_for(s);
    return tc > mma ? tc : mma;
}

template <int CIN, int COUT>
static int launch_wgrad(sg_shape s, const void* x, const void* dz, float* dw, float* db, void* scratch,
                        cudaStream_t st) {
    float* partials = static_cast<float*>(scratch);
    // bias partials after the largest weight-gradient partials either kernel writes
    float* bias_part = db ? partials + wgrad_parts_max(s) * 27 * CIN * COUT : nullptr;
    int parts, bias_parts = kBiasBlocks;
    if (g_fwd_impl == SG_CONV_TCGEN05) {
        // the tcgen05 kernel also sums the bias gradient, one partial per CTA
        parts = wgrad_tc_ctas(s);
        if (parts < 1) return -3;
        const int rc = launch_wgrad_tc<CIN, COUT>(s, x, dz, partials, bias_part, parts, st);
        if (rc) return rc;
        bias_parts = parts;
    } else {
        parts = parts_for(s);
        k_conv_wgrad<CIN, COUT><<<dim3(27, parts), kWgThreads, 0, st>>>(s, static_cast<const bf16*>(x),
                                                                         static_cast<const bf16*>(dz), partials, parts);
        if (db) {
            const int64_t voxels = (int64_t)s.batch * s.nz * s.ny * s.nx;
            k_bias_partials<<<kBiasBlocks, 256, 0, st>>>(voxels, COUT, static_cast<const bf16*>(dz), bias_part);
        }
    }
    const int n = 27 * CIN * COUT;
    k_wgrad_reduce<<<(n + 31) / 32, 256, 0, st>>>(CIN, COUT, parts, partials, dw);
    if (db) k_bias_finish<<<1, 32 * COUT, 0, st>>>(bias_parts, COUT, bias_part, db);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Valid convolution volume; an x period of 0 becomes the row (kW).
static bool shape_ok(sg_shape& s) {
    if (s.xper == 0) s.xper = kW;
    const bool per = s.xper == kW || s.xper == 32 || s.xper == 16 || s.xper == 8;
    return per && s.batch >= 1 && s.nz >= 1 && s.nx == kW && s.ny >= kRT && s.ny % kRT == 0;
}

}  // namespace sg

using namespace sg;

extern "C" {

int sg_conv3d_fwd(sg_shape s, int cin, int cout, const void* x, const void* w, const float* bias, int act,
                  int res_in, const void* add, float* z_out, void* y, void* stream) {
    Epi e{act, res_in, add, 0, z_out, 0};
    if (!x || !w || !y || !shape_ok(s) || (res_in && cin != cout)) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    if (cin == 16 && cout == 32) return launch_fwd<16, 32>(s, x, w, bias, e, y, st);
    if (cin == 32 && cout == 32) return launch_fwd<32, 32>(s, x, w, bias, e, y, st);
    if (cin == 32 && cout == 16) return launch_fwd<32, 16>(s, x, w, bias, e, y, st);
    if (cin == 16 && cout == 16) return launch_fwd<16, 16>(s, x, w, bias, e, y, st);
    return -1;
}

// Input-gradient form: y (FP32) = conv(x, w) + add (FP32, may be NULL).
int sg_conv3d_fwd_f32(sg_shape s, int cin, int cout, const void* x, const void* w, const float* add, float* y,
                      void* stream) {
    Epi e{SG_ACT_NONE, 0, add, 1, nullptr, 1};
    if (!x || !w || !y || !shape_ok(s)) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    if (cin == 16 && cout == 32) return launch_fwd<16, 32>(s, x, w, nullptr, e, y, st);
    if (cin == 32 && cout == 32) return launch_fwd<32, 32>(s, x, w, nullptr, e, y, st);
    if (cin == 32 && cout == 16) return launch_fwd<32, 16>(s, x, w, nullptr, e, y, st);
    if (cin == 16 && cout == 16) return launch_fwd<16, 16>(s, x, w, nullptr, e, y, st);
    return -1;
}

int sg_set_conv_impl(int impl) {
    if (impl != SG_CONV_MMA_SYNC && impl != SG_CONV_TCGEN05) return -1;
    const int prev = g_fwd_impl;
    g_fwd_impl = impl;
    return prev;
}

int sg_status(void* stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return -3;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_sg_status, sizeof(int)) != cudaSuccess) return -3;
    if (v) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_sg_status, &zero, sizeof(int)) != cudaSuccess) return -3;
        return -6;
    }
    return 0;
}

int sg_act_backward(int64_t n, int act, const float* dy, const float* z, void* dz, void* stream) {
    if (n < 0 || !dy || !dz || (act == SG_ACT_GELU && !z)) return -1;
    if (n == 0) return 0;
    k_act_bwd<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, act, dy, z, static_cast<bf16*>(dz));
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int sg_transpose_weights(int cin, int cout, const void* w, void* wt, void* stream) {
    if (!w || !wt || cin < 1 || cout < 1) return -1;
    const int n = 27 * cin * cout;
    k_transpose_w<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(cin, cout, static_cast<const bf16*>(w),
                                                                     static_cast<bf16*>(wt));
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int64_t sg_wgrad_scratch_bytes(sg_shape s, int cin, int cout) {
    // the weight-gradient partials of either kernel, then the bias partials
    return (wgrad_parts_max(s) * 27 * cin * cout + (int64_t)kBiasBlocks * cout) * (int64_t)sizeof(float);
}

int sg_conv3d_wgrad(sg_shape s, int cin, int cout, const void* x, const void* dz, float* dw, float* db, void* scratch,
                    void* stream) {
    if (!x || !dz || !dw || !scratch || !shape_ok(s)) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    if (cin == 16 && cout == 32) return launch_wgrad<16, 32>(s, x, dz, dw, db, scratch, st);
    if (cin == 32 && cout == 32) return launch_wgrad<32, 32>(s, x, dz, dw, db, scratch, st);
    if (cin == 32 && cout == 16) return launch_wgrad<32, 16>(s, x, dz, dw, db, scratch, st);
    if (cin == 16 && cout == 16) return launch_wgrad<16, 16>(s, x, dz, dw, db, scratch, st);
    return -1;
}

int64_t sg_reduce_scratch_bytes(int64_t n) { return (int64_t)kRedBlocks * 64 * 2 * (int64_t)sizeof(double) + 64; }

int sg_mse(int64_t voxels, int c, int nch, const void* pred, const void* target, float* loss, float* dpred,
           void* scratch, void* stream) {
    if (!pred || !target || !loss || !dpred || !scratch || nch > c || voxels < 1) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    float* partial = static_cast<float*>(scratch);
    k_mse<<<kRedBlocks, 256, 0, st>>>(voxels, c, nch, static_cast<const bf16*>(pred), static_cast<const bf16*>(target),
                                      dpred, partial);
    k_finish_mse<<<1, 32, 0, st>>>(kRedBlocks, (double)voxels * nch, partial, loss);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int sg_rel_l2(sg_shape s, int c, int nch, const void* a, const void* b, float* out, void* scratch, void* stream) {
    if (!a || !b || !out || !scratch || s.batch < 1 || s.batch > 64 || nch > c) return -1;
    const int64_t per_item = (int64_t)s.nz * s.ny * s.nx;
    k_rel_l2<<<dim3(kRedBlocks, s.batch), 256, 0, (cudaStream_t)stream>>>(
        per_item, c, nch, static_cast<const bf16*>(a), static_cast<const bf16*>(b), static_cast<double*>(scratch));
    k_finish_rel_l2<<<1, 64, 0, (cudaStream_t)stream>>>(s.batch, kRedBlocks, static_cast<const double*>(scratch), out);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int sg_adam(int64_t n, float* p, const float* g, float* m, float* v, void* p16, float lr, float beta1, float beta2,
            float eps, int t, void* stream) {
    if (!p || !g || !m || !v || t < 1 || n < 0) return -1;
    if (n == 0) return 0;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, static_cast<bf16*>(p16), lr,
                                                                           beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int sg_relabel(sg_shape s, int bytes_per_voxel, int df, int dt, const void* src, void* dst, void* stream) {
    auto log2_of = [](int v) {  // log2 of a power of two in [1, 256], else -1
        for (int l = 0; l <= 8; ++l)
            if (v == (1 << l)) return l;
        return -1;
    };
    const int lf = log2_of(df), lt = log2_of(dt), lc = log2_of(bytes_per_voxel / 16);
    auto dil_ok = [&](int l, int d) { return l >= 0 && l <= 3 && s.nz % d == 0 && s.ny % d == 0; };
    const int64_t nchunks = (int64_t)s.batch * s.nz * s.ny * kW << (lc < 0 ? 0 : lc);
    if (!src || !dst || src == dst || s.batch < 1 || s.nz < 1 || s.ny < 1 || s.nx != kW || !dil_ok(lf, df) ||
        !dil_ok(lt, dt) || bytes_per_voxel % 16 || lc < 0 || nchunks >= ((int64_t)1 << 31) || ((uintptr_t)src & 15) ||
        ((uintptr_t)dst & 15))
        return -1;
    const unsigned blocks = (unsigned)std::min<int64_t>((nchunks + 255) / 256, 152 * 16);
    k_relabel<<<blocks, 256, 0, (cudaStream_t)stream>>>((int)nchunks, s.nz, s.ny, lc, lf, lt,
                                                        static_cast<const uint4*>(src), static_cast<uint4*>(dst));
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int sg_pack_fields(sg_shape s, int item, const double* rho, const double* u, const double* theta, double theta0,
                   const float* scales, void* x, void* stream) {
    if (!rho || !u || !theta || !scales || !x || item < 0 || item >= s.batch) return -1;
    const int64_t plane = (int64_t)s.nz * s.ny * s.nx;
    k_pack<<<(unsigned)((plane + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        s, item, rho, u, theta, theta0, scales[0], scales[1], scales[2], static_cast<bf16*>(x));
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int sg_unpack_fields(sg_shape s, int item, const void* x, double theta0, const float* scales, double* rho, double* u,
                     double* theta, void* stream) {
    if (!rho || !u || !theta || !scales || !x || item < 0 || item >= s.batch) return -1;
    const int64_t n = 2 * (int64_t)s.nz * s.ny * s.nx;
    k_unpack<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        s, item, static_cast<const bf16*>(x), theta0, scales[0], scales[1], scales[2], rho, u, theta);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
