// Shared-memory-staged (TMA bulk copy) variant of the fused pull update.
//
// The grid of nodes is cut into tiles of TX consecutive x of one row
// (s, z, y).  A persistent CTA walks its tiles; for each tile, warp 0 issues
// one 1D bulk copy (cp.async.bulk, the TMA engine) per population plane: the
// plane's upwind row for that tile, widened by a 16-byte halo on each side so
// every copy starts and ends on a 16-byte boundary, with the periodic wrap at
// the row ends done as separate 16-byte pieces.  Copies land in a STAGES-deep
// ring of shared-memory buffers, each tracked by an mbarrier with a
// transaction count.  Compute threads then read the shifted neighbours with
// shared-memory loads at compile-time offsets, so there is no per-population
// global address arithmetic and the number of bytes in flight is set by the
// ring depth, not by registers.
//
// Preconditions (checked by the launcher): nx % TX == 0 and the row length in
// bytes is a multiple of 16.  Every wait on an mbarrier is bounded; on expiry
// the kernel sets bit 2 of the error word, waits (bounded) for its own copies
// in flight and returns.
#pragma once

#include "lb_common.cuh"
#include "lb_launch.h"

namespace gblb {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.b32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Spin on the phase with a cycle budget; false if the budget ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

template <class Codec, int TX_, int THREADS_, int STAGES_, int MINB_>
struct TmaCfg {
    using T = typename Codec::raw_t;
    static constexpr int TX = TX_;
    static constexpr int THREADS = THREADS_;
    static constexpr int STAGES = STAGES_;
    static constexpr int MINB = MINB_;  // CTAs per SM the register budget is sized for
    static constexpr int H = 16 / (int)sizeof(T);  // halo: 16 bytes of elements on each side
    static constexpr int ROW = TX + 2 * H;          // elements of one plane row in shared memory
    static constexpr int STAGE_ELEMS = kQ * ROW;
    static constexpr int STAGE_BYTES = STAGE_ELEMS * (int)sizeof(T);
    static constexpr int SMEM = STAGES * STAGE_BYTES + STAGES * 8 + 16;
    static constexpr int NPT = TX / THREADS;
    static_assert(TX % THREADS == 0, "TX must be a multiple of THREADS");
    static_assert((TX * sizeof(T)) % 16 == 0, "tile rows must be whole 16-byte units");
    static_assert(H >= 2, "halo must cover shifts of two cells");
};

// Tile t -> row (s, z, y) and first x.
struct TileCoord {
    int s, z, y, x0;
};

__device__ __forceinline__ TileCoord tile_coord(int64_t t, int tiles_per_row, int tx, const Dims& d) {
    TileCoord c;
    const int64_t row = t / tiles_per_row;
    c.x0 = (int)(t - row * tiles_per_row) * tx;
    c.y = (int)(row % d.ny);
    const int64_t zr = row / d.ny;
    c.z = (int)(zr % d.nz);
    c.s = (int)(zr / d.nz);
    return c;
}

template <class Codec, bool PROJECT, class Cfg>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MINB) k_step_tma(const typename Codec::raw_t* __restrict__ src,
                                                           typename Codec::raw_t* __restrict__ dst, Dims d,
                                                           Consts<typename Codec::R> K, typename Codec::R tb,
                                                           int* __restrict__ err, long long wait_limit) {
    using R = typename Codec::R;
    using T = typename Codec::raw_t;
    constexpr int TX = Cfg::TX, H = Cfg::H, ROW = Cfg::ROW, STAGES = Cfg::STAGES;
    extern __shared__ __align__(128) unsigned char smem[];
    T* stage_base = reinterpret_cast<T*>(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
    int* flag = reinterpret_cast<int*>(bars + STAGES);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool producer = tid < 32;
    const int tiles_per_row = d.nx / TX;
    const int64_t ntiles = d.rows * tiles_per_row;
    const int64_t nxy = (int64_t)d.nx * d.ny;
    const int64_t my_tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) mbar_init(smem_u32(&bars[i]), 1);
        *flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // warp 0: issue the 41 plane copies of this CTA's k-th tile into stage k % STAGES
    auto issue = [&](int64_t k) {
        const int st = (int)(k % STAGES);
        const TileCoord tc = tile_coord(blockIdx.x + k * gridDim.x, tiles_per_row, TX, d);
        const uint32_t bar = smem_u32(&bars[st]);
        fence_proxy_async_smem();
        if (lane == 0) mbar_arrive_expect_tx(bar, Cfg::STAGE_BYTES);
        __syncwarp();
        const bool left = tc.x0 == 0;
        const bool right = tc.x0 + TX == d.nx;
        constexpr uint32_t HB = H * sizeof(T);  // 16 bytes
        for (int i = lane; i < kQ; i += 32) {
            const Vel c = c_vel.v[i];
            int sp, dy, dz;
            if (c.shell == 5) {
                sp = 1 - tc.s;
                dy = c.y > 0 ? 1 - tc.s : -tc.s;
                dz = c.z > 0 ? 1 - tc.s : -tc.s;
            } else {
                sp = tc.s;
                dy = c.y / 2;
                dz = c.z / 2;
            }
            const int ys = wrap(tc.y - dy, d.ny), zs = wrap(tc.z - dz, d.nz);
            const T* rowp = src + ((int64_t)sp * kQ + i) * d.plane + (int64_t)zs * nxy + (int64_t)ys * d.nx;
            const uint32_t dsm = smem_u32(stage_base + (int64_t)st * Cfg::STAGE_ELEMS + i * ROW);
            // shared row j holds global x = (x0 - H + j) mod nx
            if (!left && !right) {
                bulk_g2s(dsm, rowp + tc.x0 - H, (uint32_t)(ROW * sizeof(T)), bar);
            } else if (left && !right) {
                bulk_g2s(dsm, rowp + d.nx - H, HB, bar);
                bulk_g2s(dsm + HB, rowp, (uint32_t)((TX + H) * sizeof(T)), bar);
            } else if (!left && right) {
                bulk_g2s(dsm, rowp + tc.x0 - H, (uint32_t)((TX + H) * sizeof(T)), bar);
                bulk_g2s(dsm + (uint32_t)((TX + H) * sizeof(T)), rowp, HB, bar);
            } else {  // one tile spans the whole row
                bulk_g2s(dsm, rowp + d.nx - H, HB, bar);
                bulk_g2s(dsm + HB, rowp, (uint32_t)(TX * sizeof(T)), bar);
                bulk_g2s(dsm + HB + (uint32_t)(TX * sizeof(T)), rowp, HB, bar);
            }
        }
    };

    if (producer)
        for (int64_t k = 0; k < STAGES - 1 && k < my_tiles; ++k) issue(k);

    constexpr R inv_scale = R(1.0 / Codec::kScale);
    const R tbs = tb * R(Codec::kScale);
    const R omb = R(1) - tb;
    int64_t k = 0;
    for (; k < my_tiles; ++k) {
        const int st = (int)(k % STAGES);
        if (tid == 0 && !mbar_wait_bounded(smem_u32(&bars[st]), (uint32_t)((k / STAGES) & 1), wait_limit)) *flag = 1;
        // every thread has finished tile k-1, so its stage may be refilled
        if (__syncthreads_or(tid == 0 ? *flag : 0)) break;
        if (producer && k + STAGES - 1 < my_tiles) issue(k + STAGES - 1);

        const TileCoord tc = tile_coord(blockIdx.x + k * gridDim.x, tiles_per_row, TX, d);
        const T* sb = stage_base + (int64_t)st * Cfg::STAGE_ELEMS;
        T* outrow = dst + (int64_t)tc.s * kQ * d.plane + (int64_t)tc.z * nxy + (int64_t)tc.y * d.nx + tc.x0;
        const int s = tc.s;
#pragma unroll
        for (int j = 0; j < Cfg::NPT; ++j) {
            const int xl = tid + j * Cfg::THREADS;
            // shared index of plane I's upwind value: xl + H - dx_I
            auto vget = [&](auto I) -> R {
                constexpr Vel c = vel(I);
                if constexpr (c.shell == 5) {
                    // dx = 1 - s for a +1/2 component, -s for -1/2
                    return Codec::value(sb[I * ROW + xl + (c.x > 0 ? H - 1 : H) + s]);
                } else {
                    return Codec::value(sb[I * ROW + xl + H - c.x / 2]);
                }
            };
            const NodeMoments<R> m = moments_from<R>([&](auto I) { return Codec::dev(vget(I), K.w[vel(I).shell] * inv_scale); });
            const NodeState<R> ns = state_from_moments(m, K);
            if (!state_ok(ns)) atomicOr(err, 1);
            T* out = outrow + xl;
            equilibrium_relax_g<Codec, PROJECT>(ns, K, tbs, omb, vget,
                                                [&](auto I, R val) { out[(int64_t)I * d.plane] = Codec::to_raw(val); });
        }
    }
    if (k < my_tiles) {
        // a wait ran out: report, let this CTA's copies in flight land (bounded), leave
        if (tid == 0) {
            atomicOr(err, 2);
            const int64_t last = k + STAGES - 1 < my_tiles ? k + STAGES - 1 : my_tiles;
            for (int64_t kk = k; kk < last; ++kk)
                mbar_wait_bounded(smem_u32(&bars[kk % STAGES]), (uint32_t)((kk / STAGES) & 1), wait_limit);
        }
        __syncthreads();
    }
}

}  // namespace gblb
