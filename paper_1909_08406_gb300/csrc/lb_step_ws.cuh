// Warp-specialised, TMA-staged step kernel (FP32 arithmetic; FP32/FP16/BF16
// storage).
//
// Tile: TX consecutive x of two rows (y, y + 1) of one (s, z) plane.  Warp 0
// is the producer: for each of its CTA's tiles it fetches, per population
// plane, the two upwind rows of the tile (widened by a 16-byte halo, periodic
// wrap done as extra 16-byte pieces) with 1D cp.async.bulk copies into a
// STAGES-deep shared-memory ring.  Each stage has a "full" mbarrier (producer
// arrival with the byte count; the copies complete the transactions) and an
// "empty" mbarrier (one arrival per consumer warp).  Warps 1..CW are
// consumers: each thread updates the nodes (x, y) and (x, y + 1) with packed
// FP32x2 arithmetic, reading the shifted neighbours from shared memory at
// compile-time offsets, and stores the 82 results directly.  No block-wide
// barrier is taken inside the loop.  Every mbarrier wait is bounded; on
// expiry the kernel sets bit 2 of the error word, lets its own copies land
// (bounded) and returns.
#pragma once

#include "lb_kernels.cuh"
#include "lb_step_tma.cuh"

namespace gblb {

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Shared-memory loads the compiler may not merge: the consumers read each staged value
// once per pass instead of keeping 41 values live in registers between the passes.
template <class T>
__device__ __forceinline__ T lds_keep(uint32_t addr);
template <>
__device__ __forceinline__ __half lds_keep<__half>(uint32_t addr) {
    unsigned short v;
    asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(addr));
    return __ushort_as_half(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 lds_keep<__nv_bfloat16>(uint32_t addr) {
    unsigned short v;
    asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(addr));
    return __ushort_as_bfloat16(v);
}
template <>
__device__ __forceinline__ float lds_keep<float>(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

template <class Codec, int TX_, int CW_, int STAGES_, int MINB_>
struct WsCfg {
    using T = typename Codec::raw_t;
    static constexpr int TX = TX_;            // x per tile (= consumer threads)
    static constexpr int CW = CW_;            // consumer warps
    static constexpr int THREADS = 32 * (CW + 1);
    static constexpr int STAGES = STAGES_;
    static constexpr int MINB = MINB_;
    static constexpr int H = 16 / (int)sizeof(T);
    static constexpr int ROW = TX + 2 * H;               // elements per staged row
    static constexpr int STAGE_ELEMS = kQ * 2 * ROW;      // [plane][row 0/1][ROW]
    static constexpr int STAGE_BYTES = STAGE_ELEMS * (int)sizeof(T);
    static constexpr int SMEM = STAGES * STAGE_BYTES + 2 * STAGES * 8 + 16;
    static_assert(TX == 32 * CW, "one consumer thread per x");
    static_assert((TX * sizeof(T)) % 16 == 0, "tile rows must be whole 16-byte units");
};

template <class Codec, bool PROJECT, class Cfg>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MINB) k_step_ws(const typename Codec::raw_t* __restrict__ src,
                                                                    typename Codec::raw_t* __restrict__ dst, Dims d,
                                                                    Consts<float> K, float tb, int* __restrict__ err,
                                                                    long long wait_limit) {
    using T = typename Codec::raw_t;
    using C2 = Codec2<Codec>;
    constexpr int TX = Cfg::TX, H = Cfg::H, ROW = Cfg::ROW, STAGES = Cfg::STAGES;
    extern __shared__ __align__(128) unsigned char smem[];
    T* stage_base = reinterpret_cast<T*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    int* flag = reinterpret_cast<int*>(empty + STAGES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_per_row = d.nx / TX;
    const int nyh = d.ny >> 1;
    const int64_t ntiles = d.rows / 2 * tiles_per_row;  // row pairs x tiles
    const int64_t my_tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
    const uint32_t plane = (uint32_t)d.plane;

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), Cfg::CW);
        }
        *flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // tile t -> (s, z, y pair, x0)
    auto coord = [&](int64_t t, int& s, int& z, int& y, int& x0) {
        const int64_t rp = t / tiles_per_row;
        x0 = (int)(t - rp * tiles_per_row) * TX;
        y = 2 * (int)(rp % nyh);
        const int64_t zr = rp / nyh;
        z = (int)(zr % d.nz);
        s = (int)(zr / d.nz);
    };

    if (warp == 0) {
        // ---------------- producer ----------------
        int64_t k = 0;
        for (; k < my_tiles; ++k) {
            const int st = (int)(k % STAGES);
            const uint32_t n = (uint32_t)(k / STAGES);
            if (k >= STAGES) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_bounded(smem_u32(&empty[st]), (n - 1) & 1, wait_limit);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) {
                        atomicOr(err, 2);
                        atomicExch(flag, 1);
                    }
                    break;
                }
            }
            if (*reinterpret_cast<volatile int*>(flag)) break;
            int s, z, y, x0;
            coord(blockIdx.x + k * gridDim.x, s, z, y, x0);
            const uint32_t fb = smem_u32(&full[st]);
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(fb, Cfg::STAGE_BYTES);
            __syncwarp();
            const bool left = x0 == 0, right = x0 + TX == d.nx;
            constexpr uint32_t HB = H * sizeof(T);
            for (int item = lane; item < 2 * kQ; item += 32) {
                const int i = item >> 1, r = item & 1;
                const Vel c = c_vel.v[i];
                int sp, dy, dz;
                if (c.shell == 5) {
                    sp = 1 - s;
                    dy = c.y > 0 ? 1 - s : -s;
                    dz = c.z > 0 ? 1 - s : -s;
                } else {
                    sp = s;
                    dy = c.y / 2;
                    dz = c.z / 2;
                }
                const int ys = wrap(y + r - dy, d.ny), zs = wrap(z - dz, d.nz);
                const T* rowp = src + ((size_t)sp * kQ + i) * d.plane + (size_t)zs * nxy + (size_t)ys * nx;
                const uint32_t dsm = smem_u32(stage_base + (size_t)st * Cfg::STAGE_ELEMS + (i * 2 + r) * ROW);
                if (!left && !right) {
                    bulk_g2s(dsm, rowp + x0 - H, (uint32_t)(ROW * sizeof(T)), fb);
                } else if (left && !right) {
                    bulk_g2s(dsm, rowp + d.nx - H, HB, fb);
                    bulk_g2s(dsm + HB, rowp, (uint32_t)((TX + H) * sizeof(T)), fb);
                } else if (!left && right) {
                    bulk_g2s(dsm, rowp + x0 - H, (uint32_t)((TX + H) * sizeof(T)), fb);
                    bulk_g2s(dsm + (uint32_t)((TX + H) * sizeof(T)), rowp, HB, fb);
                } else {
                    bulk_g2s(dsm, rowp + d.nx - H, HB, fb);
                    bulk_g2s(dsm + HB, rowp, (uint32_t)(TX * sizeof(T)), fb);
                    bulk_g2s(dsm + HB + (uint32_t)(TX * sizeof(T)), rowp, HB, fb);
                }
            }
        }
        // let every issued copy land before the CTA can exit (tiles k-STAGES+1 .. k-1 at most in flight)
        if (lane == 0) {
            const int64_t first = k > STAGES ? k - STAGES : 0;
            for (int64_t kk = first; kk < k; ++kk)
                mbar_wait_bounded(smem_u32(&full[kk % STAGES]), (uint32_t)((kk / STAGES) & 1), wait_limit);
        }
    } else {
        // ---------------- consumers ----------------
        const int xl = tid - 32;
        constexpr float inv_scale = (float)(1.0 / Codec::kScale);
        const F2 tbs(tb * (float)Codec::kScale), omb(1.f - tb);
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int st = (int)(k % STAGES);
            if (!mbar_wait_bounded(smem_u32(&full[st]), (uint32_t)((k / STAGES) & 1), wait_limit)) {
                if (lane == 0) {
                    atomicOr(err, 2);
                    atomicExch(flag, 1);
                }
                break;
            }
            int s, z, y, x0;
            coord(blockIdx.x + k * gridDim.x, s, z, y, x0);
            const uint32_t sbu = smem_u32(stage_base + (size_t)st * Cfg::STAGE_ELEMS);
            // shared index of plane I, row r: (2 I + r) ROW + xl + H - dx_I; values are read from the
            // ring in both passes (moments, relaxation) instead of being held in registers
            auto vget = [&](auto I) {
                constexpr Vel c = vel(I);
                int off;
                if constexpr (c.shell == 5)
                    off = xl + (c.x > 0 ? H - 1 : H) + s;
                else
                    off = xl + H - c.x / 2;
                const uint32_t a = sbu + (uint32_t)(((2 * I) * ROW + off) * (int)sizeof(T));
                return F2(Codec::value(lds_keep<T>(a)), Codec::value(lds_keep<T>(a + ROW * (int)sizeof(T))));
            };
            const NodeMoments<F2> m =
                moments_from<F2>([&](auto I) { return C2::dev(vget(I), F2(K.w[vel(I).shell] * inv_scale)); });
            const NodeState<F2> ns = state_from_moments(m, K);
            if (!state_ok(ns)) atomicOr(err, 1);
            T* outa = dst + (size_t)s * kQ * d.plane + ((uint32_t)z * nxy + (uint32_t)y * nx + (uint32_t)(x0 + xl));
            equilibrium_relax_g<C2, PROJECT>(ns, K, tbs, omb, vget, [&](auto I, F2 val) {
                T* p = outa + (size_t)I * plane;
                p[0] = Codec::to_raw(val.v.x);
                p[nx] = Codec::to_raw(val.v.y);
            });
            // this warp is done with the stage: release it to the producer
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
        }
    }
}

}  // namespace gblb
