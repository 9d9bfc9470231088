// Kernel templates of the RD3Q41 solver.  Each translation unit that includes
// this header instantiates the kernels for the codecs it needs (FP32-family
// kernels are compiled with double-precision-use warnings enabled).
#pragma once

#include "lb_common.cuh"
#include "lb_launch.h"

namespace gblb {

constexpr int kStepThreads = 128;

// Load paths: the read-only (non-coherent) path for kernels whose inputs no
// thread of the same launch writes, and L2-coherent loads for persistent
// kernels that read, after a grid barrier, what other CTAs wrote.
struct LoadNC {
    template <class T>
    static __device__ __forceinline__ T load(const T* p) {
        return __ldg(p);
    }
};
struct LoadCG {
    template <class T>
    static __device__ __forceinline__ T load(const T* p) {
        return __ldcg(p);
    }
};
// Fused pull update (Sec. II) of one node (s, z, y, x): gather f*_i(x - c_i, t)
// for all 41 velocities, compute the moments, the equilibrium and the BGK
// relaxation, and write the 41 post-collision values.  Integer links stay on
// the sub-lattice (shifts 0, +-1, +-2 cells); the bcc-1/2 links come from the
// other sub-lattice: for A (s = 0) a component +1/2 reads cell r - 1 and -1/2
// reads cell r; for B (s = 1) +1/2 reads cell r and -1/2 reads cell r + 1.
// SR: BF16 storage with the stochastic store of lb_common.cuh, step key sr_key.
template <class Codec, int EQ, class Ld = LoadNC, bool SR = false>
__device__ __forceinline__ void step_node(const typename Codec::raw_t* __restrict__ src,
                                          typename Codec::raw_t* __restrict__ dst, const Dims& d,
                                          const Consts<typename Codec::R>& K, typename Codec::R tb,
                                          int* __restrict__ err, int s, int z, int y, int x, uint32_t sr_key = 0) {
    using R = typename Codec::R;
    using T = typename Codec::raw_t;
    const int64_t nxy = (int64_t)d.nx * d.ny;

    // coordinate / offset of the upwind cell for a shift delta = k - 2 (source = x - delta)
    int xs[5];
    int64_t yo[5], zo[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        xs[k] = wrap(x - (k - 2), d.nx);
        yo[k] = (int64_t)wrap(y - (k - 2), d.ny) * d.nx;
        zo[k] = (int64_t)wrap(z - (k - 2), d.nz) * nxy;
    }
    // half links: component +1/2 has delta = 1 - s, component -1/2 has delta = -s
    const int hxp = s ? xs[2] : xs[3], hxm = s ? xs[1] : xs[2];
    const int64_t hyp = s ? yo[2] : yo[3], hym = s ? yo[1] : yo[2];
    const int64_t hzp = s ? zo[2] : zo[3], hzm = s ? zo[1] : zo[2];

    const T* same = src + (int64_t)s * kQ * d.plane;
    const T* other = src + (int64_t)(1 - s) * kQ * d.plane;

    R v[kQ];
    static_for<kQ>([&](auto I) {
        constexpr Vel c = vel(I);
        if constexpr (c.shell == 5) {
            const int64_t off = (c.z > 0 ? hzp : hzm) + (c.y > 0 ? hyp : hym) + (c.x > 0 ? hxp : hxm);
            v[I] = Codec::value(Ld::load(other + (int64_t)I * d.plane + off));
        } else {
            const int64_t off = zo[c.z / 2 + 2] + yo[c.y / 2 + 2] + xs[c.x / 2 + 2];
            v[I] = Codec::value(Ld::load(same + (int64_t)I * d.plane + off));
        }
    });

    R dv[kQ];
    constexpr R inv_scale = R(1.0 / Codec::kScale);
    static_for<kQ>([&](auto I) { dv[I] = Codec::dev(v[I], K.w[vel(I).shell] * inv_scale); });
    const NodeMoments<R> m = moments_from_dev(dv);
    const NodeState<R> st = state_from_moments(m, K);
    bool ok = state_ok(st);

    const int64_t qn = (int64_t)z * nxy + (int64_t)y * d.nx + x;
    T* out = dst + (int64_t)s * kQ * d.plane + qn;
    if constexpr (SR) {
        const uint32_t q = (uint32_t)((int64_t)s * d.plane + qn);
        const uint32_t s0 = pcg_hash(sr_key ^ (q >> 1));
        equilibrium_relax<Codec, EQ>(st, K, tb * R(Codec::kScale), R(1) - tb, v,
                                     [&](auto I, R val) {
                                         const uint32_t w = sr_word<decltype(I)::value>(s0);
                                         out[(int64_t)I * d.plane] = sr_bf16(val, (q & 1u) ? (w >> 16) : (w & 0xFFFFu));
                                     },
                                     ok);
    } else {
        equilibrium_relax<Codec, EQ>(st, K, tb * R(Codec::kScale), R(1) - tb, v,
                                     [&](auto I, R val) { out[(int64_t)I * d.plane] = Codec::to_raw(val); }, ok);
    }
    if (!ok) atomicOr(err, 1);
}

// Direct-load step kernel.  Grid: blockIdx.x = row (s, z, y),
// blockIdx.y * blockDim.x + threadIdx.x = x.  EQ: equilibrium kind (see
// equilibrium_relax).
template <class Codec, int EQ>
__global__ void __launch_bounds__(kStepThreads) k_step(const typename Codec::raw_t* __restrict__ src,
                                                       typename Codec::raw_t* __restrict__ dst, Dims d,
                                                       Consts<typename Codec::R> K, typename Codec::R tb,
                                                       int* __restrict__ err) {
    const int x = blockIdx.y * blockDim.x + threadIdx.x;
    if (x >= d.nx) return;
    const int64_t row = blockIdx.x;
    const int y = (int)(row % d.ny);
    const int64_t zr = row / d.ny;
    const int z = (int)(zr % d.nz);
    const int s = (int)(zr / d.nz);
    step_node<Codec, EQ>(src, dst, d, K, tb, err, s, z, y, x);
}

template <class Codec, bool PROJECT, class Ld>
__device__ __forceinline__ void step_node2(const typename Codec::raw_t* __restrict__ src,
                                           typename Codec::raw_t* __restrict__ dst, const Dims& d,
                                           const Consts<float>& K, float tb, int* __restrict__ err, int s, int z,
                                           int y, int x);

// k_step with the stochastic BF16 store (series equilibrium with the momentum projection).
template <class Codec>
__global__ void __launch_bounds__(kStepThreads) k_step_sr(const typename Codec::raw_t* __restrict__ src,
                                                          typename Codec::raw_t* __restrict__ dst, Dims d,
                                                          Consts<typename Codec::R> K, typename Codec::R tb,
                                                          int* __restrict__ err, uint32_t sr_key) {
    const int x = blockIdx.y * blockDim.x + threadIdx.x;
    if (x >= d.nx) return;
    const int64_t row = blockIdx.x;
    const int y = (int)(row % d.ny);
    const int64_t zr = row / d.ny;
    const int z = (int)(zr % d.nz);
    const int s = (int)(zr / d.nz);
    step_node<Codec, 1, LoadNC, true>(src, dst, d, K, tb, err, s, z, y, x, sr_key);
}

// Two-rows-per-thread direct-load step kernel (FP32 arithmetic, any storage
// except FP64): each thread updates nodes (s, z, y, x) and (s, z, y + 1, x)
// with packed FP32x2 arithmetic.  Addresses are formed from 32-bit in-plane
// offsets (the host guarantees nx * ny * nz < 2^32) plus plane * I.  Blocks
// are numbered chunk-fastest, so the CTAs covering one row segment run
// together and the sectors they share at chunk and wrap boundaries stay in
// L2.  Requires ny even.  Grid: (nz * ny / 2 * 2 sub-lattices) * chunks blocks.
template <class Codec, bool PROJECT, int MINB>
__global__ void __launch_bounds__(kStepThreads, MINB) k_step2(const typename Codec::raw_t* __restrict__ src,
                                                        typename Codec::raw_t* __restrict__ dst, Dims d,
                                                        Consts<float> K, float tb, int* __restrict__ err,
                                                        int chunks) {
    const int64_t t = blockIdx.x;
    const int64_t rp = t / chunks;
    const int x = (int)(t - rp * chunks) * blockDim.x + threadIdx.x;
    if (x >= d.nx) return;
    const int nyh = d.ny >> 1;
    const int y = 2 * (int)(rp % nyh);
    const int64_t zr = rp / nyh;
    const int z = (int)(zr % d.nz);
    const int s = (int)(zr / d.nz);
    step_node2<Codec, PROJECT, LoadNC>(src, dst, d, K, tb, err, s, z, y, x);
}

// Nodes (s, z, y, x) and (s, z, y + 1, x) (y even), packed FP32x2 arithmetic; see k_step2.
template <class Codec, bool PROJECT, class Ld>
__device__ __forceinline__ void step_node2(const typename Codec::raw_t* __restrict__ src,
                                           typename Codec::raw_t* __restrict__ dst, const Dims& d,
                                           const Consts<float>& K, float tb, int* __restrict__ err, int s, int z,
                                           int y, int x) {
    using T = typename Codec::raw_t;
    using C2 = Codec2<Codec>;
    const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
    const uint32_t plane = (uint32_t)d.plane;

    // source coordinates: x - delta for delta = k - 2; rows y + k - 2 for k = 0..5 (covers
    // y - delta for the first node and y + 1 - delta for the second); planes z - delta
    uint32_t xs[5], yo[6], zo[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        xs[k] = (uint32_t)wrap(x - (k - 2), d.nx);
        zo[k] = (uint32_t)wrap(z - (k - 2), d.nz) * nxy;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) yo[k] = (uint32_t)wrap(y + k - 2, d.ny) * nx;
    // half links: delta = 1 - s for a +1/2 component, -s for -1/2; the row index is 2 - delta
    const uint32_t hxp = s ? xs[2] : xs[3], hxm = s ? xs[1] : xs[2];
    const uint32_t hzp = s ? zo[2] : zo[3], hzm = s ? zo[1] : zo[2];
    const int kyp = 1 + s, kym = 2 + s;  // 2 - delta for +1/2 and -1/2

    const T* same = src + (size_t)s * kQ * d.plane;
    const T* other = src + (size_t)(1 - s) * kQ * d.plane;

    // the two nodes' stored values stay packed (one register per population for 16-bit
    // storage) and are widened to FP32 where they are used
    typename Codec::pair_t pv[kQ];
    static_for<kQ>([&](auto I) {
        constexpr Vel c = vel(I);
        uint32_t oa, ob;
        const T* base;
        if constexpr (c.shell == 5) {
            const uint32_t xz = (c.z > 0 ? hzp : hzm) + (c.x > 0 ? hxp : hxm);
            const int ky = c.y > 0 ? kyp : kym;
            oa = xz + yo[ky];
            ob = xz + yo[ky + 1];
            base = other;
        } else {
            const uint32_t xz = zo[c.z / 2 + 2] + xs[c.x / 2 + 2];
            oa = xz + yo[2 - c.y / 2];
            ob = xz + yo[3 - c.y / 2];
            base = same;
        }
        const T* p = base + (size_t)I * plane;
        pv[I] = Codec::pack2(Ld::load(p + oa), Ld::load(p + ob));
    });
    auto vget = [&](auto I) { return F2(Codec::unpack2(pv[I])); };

    constexpr float inv_scale = (float)(1.0 / Codec::kScale);
    const NodeMoments<F2> m = moments_from<F2>([&](auto I) { return C2::dev(vget(I), F2(K.w[vel(I).shell] * inv_scale)); });
    const NodeState<F2> st = state_from_moments(m, K);
    if (!state_ok(st)) atomicOr(err, 1);

    T* outa = dst + (size_t)s * kQ * d.plane + ((uint32_t)z * nxy + (uint32_t)y * nx + (uint32_t)x);
    equilibrium_relax_g<C2, PROJECT>(st, K, F2(tb * (float)Codec::kScale), F2(1.f - tb), vget,
                                     [&](auto I, F2 val) {
                                         T* p = outa + (size_t)I * plane;
                                         p[0] = Codec::to_raw(val.v.x);
                                         p[nx] = Codec::to_raw(val.v.y);
                                     });
}

// Two x-adjacent nodes per thread (16-bit storage): nodes (s, z, y, x) and
// (s, z, y, x + 1), x even, packed FP32x2 arithmetic.  Each plane is read as
// aligned pairs of 16-bit values: one 32-bit load when the plane's x shift is
// even, two loads and a byte permute when it is odd; the two results of a
// plane are written with one 32-bit store.
//
// A block covers one chunk of x for `rpb` consecutive rows (s, z, y), y
// fastest, and each thread loads a row's 41 pairs at the start of that row
// (MODE below says how the next row is brought closer meanwhile).  Requires
// nx even and nx * ny * nz < 2^32.
template <class Codec>
struct RowAddr2x {
    using T = typename Codec::raw_t;
    const T* same;   // population 0 of the node's own sub-lattice
    const T* other;  // population 0 of the other sub-lattice
    uint32_t yo[5], zo[5];
    uint32_t hyp, hym, hzp, hzm;
    int s;
    __device__ __forceinline__ void set(const T* src, const Dims& d, int s_, int z, int y) {
        s = s_;
        const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            yo[k] = (uint32_t)wrap(y - (k - 2), d.ny) * nx;
            zo[k] = (uint32_t)wrap(z - (k - 2), d.nz) * nxy;
        }
        // half links: delta = 1 - s for a +1/2 component, -s for -1/2
        hyp = s ? yo[2] : yo[3];
        hym = s ? yo[1] : yo[2];
        hzp = s ? zo[2] : zo[3];
        hzm = s ? zo[1] : zo[2];
        same = src + (size_t)s * kQ * d.plane;
        other = src + (size_t)(1 - s) * kQ * d.plane;
    }
};

// The pair of upwind values of population I for the nodes x, x + 1 of the row
// described by `a` (source x - delta for a shift delta in {-2, ..., 2}).
template <class Codec, int I>
__device__ __forceinline__ typename Codec::pair_t load_pair2x(const RowAddr2x<Codec>& a, uint32_t plane,
                                                              uint32_t xm, uint32_t x0, uint32_t xq) {
    using T = typename Codec::raw_t;
    using P = typename Codec::pair_t;
    constexpr Vel c = vel(I);
    auto ld = [&](const T* p, uint32_t off) { return LoadNC::load(reinterpret_cast<const P*>(p + off)); };
    auto pair_at = [&](const T* p, int dx) -> P {
        switch (dx) {
            case 2: return ld(p, xm);
            case 1: return Codec::straddle(ld(p, xm), ld(p, x0));
            case 0: return ld(p, x0);
            case -1: return Codec::straddle(ld(p, x0), ld(p, xq));
            default: return ld(p, xq);
        }
    };
    if constexpr (c.shell == 5) {
        const T* p = a.other + (size_t)I * plane + ((c.z > 0 ? a.hzp : a.hzm) + (c.y > 0 ? a.hyp : a.hym));
        if constexpr (c.x > 0)
            return a.s ? pair_at(p, 0) : pair_at(p, 1);
        else
            return a.s ? pair_at(p, -1) : pair_at(p, 0);
    } else {
        const T* p = a.same + (size_t)I * plane + (a.zo[c.z / 2 + 2] + a.yo[c.y / 2 + 2]);
        return pair_at(p, c.x / 2);
    }
}

// Prefetch into L2 the part of population I's source row that the nodes
// [xa, xb) of the row (s, z, y) will read (x - 2 .. x + 2, not wrapped),
// trimmed inward to whole 16-byte units of that row.
template <class Codec>
__device__ __forceinline__ void prefetch_row_l2(const typename Codec::raw_t* src, const Dims& d, int I, int s, int z,
                                                int y, int xa, int xb) {
    using T = typename Codec::raw_t;
    const Vel c = c_vel.v[I];
    int sp, dz, dy;
    if (c.shell == 5) {  // half link: delta = 1 - s for +1/2, -s for -1/2; other sub-lattice
        sp = 1 - s;
        dz = c.z > 0 ? 1 - s : -s;
        dy = c.y > 0 ? 1 - s : -s;
    } else {
        sp = s;
        dz = c.z / 2;
        dy = c.y / 2;
    }
    const int zz = wrap(z - dz, d.nz), yy = wrap(y - dy, d.ny);
    const int lo = max(xa - 2, 0), hi = min(xb + 2, d.nx);
    const T* row = src + ((size_t)sp * kQ + I) * d.plane + ((size_t)zz * d.ny + yy) * d.nx;
    const uintptr_t b0 = ((uintptr_t)(row + lo) + 15) & ~(uintptr_t)15;
    const uintptr_t b1 = ((uintptr_t)(row + hi)) & ~(uintptr_t)15;
    if (b1 > b0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"((uint32_t)(b1 - b0)) : "memory");
}

// How a block of the x-pair kernel gets a row's upwind values:
// MODE 0: direct loads at the start of the row.
// MODE 2: as MODE 0, plus an L2 bulk prefetch of the next row's source rows
//         (one per population, by threads 0..40; a block of only 32 threads,
//         on a narrow grid, prefetches its first 32 populations) at the start
//         of the current row, so that the next row's loads hit in L2.
// SR: BF16 storage with the stochastic store of lb_common.cuh, step key sr_key (one word per
// population and x pair).
template <class Codec, bool PROJECT, int MINB, int MODE, bool SR = false>
__global__ void __launch_bounds__(kStepThreads, MINB) k_step2x(const typename Codec::raw_t* __restrict__ src,
                                                         typename Codec::raw_t* __restrict__ dst, Dims d,
                                                         Consts<float> K, float tb, int* __restrict__ err,
                                                         int chunks, int rpb, uint32_t sr_key) {
    using T = typename Codec::raw_t;
    using P = typename Codec::pair_t;
    using C2 = Codec2<Codec>;
    const uint32_t t = blockIdx.x;
    const uint32_t grp = t / (uint32_t)chunks;
    const int chunk = (int)(t - grp * (uint32_t)chunks);
    const int x = 2 * (chunk * (int)blockDim.x + (int)threadIdx.x);
    const int xa = 2 * chunk * (int)blockDim.x, xb = min(xa + 2 * (int)blockDim.x, d.nx);
    const uint32_t r0 = grp * (uint32_t)rpb;
    const uint32_t r1 = min(r0 + (uint32_t)rpb, (uint32_t)d.rows);
    int y = (int)(r0 % (uint32_t)d.ny);
    const uint32_t zr = r0 / (uint32_t)d.ny;
    int z = (int)(zr % (uint32_t)d.nz);
    int s = (int)(zr / (uint32_t)d.nz);
    const bool active = x < d.nx;
    if (!active && (MODE != 2 || threadIdx.x >= kQ)) return;  // threads < 41 issue prefetches
    const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
    const uint32_t plane = (uint32_t)d.plane;

    // aligned pair starts: x - 2, x, x + 2 (periodic; nx even keeps them even)
    const uint32_t xm = (uint32_t)wrap(x - 2, d.nx), x0 = (uint32_t)x, xq = (uint32_t)wrap(x + 2, d.nx);

    P pv[kQ];
    auto vget = [&](auto I) { return F2(Codec::unpack2(pv[I])); };
    constexpr float inv_scale = (float)(1.0 / Codec::kScale);

    for (uint32_t r = r0; r < r1; ++r) {
        // the next row, in (s, z, y) order
        int yn = y + 1, zn = z, sn = s;
        if (yn == d.ny) {
            yn = 0;
            if (++zn == d.nz) {
                zn = 0;
                ++sn;
            }
        }
        const bool more = r + 1 < r1;
        if constexpr (MODE == 2) {
            if (more && threadIdx.x < kQ) prefetch_row_l2<Codec>(src, d, (int)threadIdx.x, sn, zn, yn, xa, xb);
            if (!active) {
                s = sn;
                z = zn;
                y = yn;
                continue;
            }
        }
        {
            RowAddr2x<Codec> a;
            a.set(src, d, s, z, y);
            static_for<kQ>([&](auto I) { pv[I] = load_pair2x<Codec, I>(a, plane, xm, x0, xq); });
        }

        const NodeMoments<F2> m =
            moments_from<F2>([&](auto I) { return C2::dev(vget(I), F2(K.w[vel(I).shell] * inv_scale)); });
        const NodeState<F2> st = state_from_moments(m, K);
        if (!state_ok(st)) atomicOr(err, 1);

        P* outp = reinterpret_cast<P*>(dst + (size_t)s * kQ * d.plane + ((uint32_t)z * nxy + (uint32_t)y * nx + x0));
        if constexpr (SR) {
            const uint32_t q = (uint32_t)s * plane + (uint32_t)z * nxy + (uint32_t)y * nx + x0;
            const uint32_t s0 = pcg_hash(sr_key ^ (q >> 1));
            equilibrium_relax_g<C2, PROJECT>(st, K, F2(tb * (float)Codec::kScale), F2(1.f - tb), vget,
                                             [&](auto I, F2 val) {
                                                 outp[(size_t)I * (plane / 2)] =
                                                     sr_bf16x2(val.v, sr_word<decltype(I)::value>(s0));
                                             });
        } else {
            equilibrium_relax_g<C2, PROJECT>(st, K, F2(tb * (float)Codec::kScale), F2(1.f - tb), vget,
                                             [&](auto I, F2 val) { outp[(size_t)I * (plane / 2)] = Codec::to_raw2(val.v); });
        }
        s = sn;
        z = zn;
        y = yn;
    }
}

// Populations = equilibrium of the given float64 fields, for nodes
// q in [q0, q0 + count), q = s * plane + (z * ny + y) * nx + x.  Field
// pointers are indexed by q - q0 (u component c at c * ustride + q - q0).
template <class Codec, int EQ>
__global__ void __launch_bounds__(256) k_init(typename Codec::raw_t* __restrict__ dst, Dims d, Consts<typename Codec::R> K,
                                              double theta0, int64_t q0, int64_t count, const double* __restrict__ rho,
                                              const double* __restrict__ u, int64_t ustride,
                                              const double* __restrict__ theta, int* __restrict__ err) {
    using R = typename Codec::R;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int64_t q = q0 + k;
    const int s = q >= d.plane;
    const int64_t node = q - s * d.plane;
    NodeState<R> st;
    st.drho = (R)(rho[k] - 1.0);
    st.rho = (R)rho[k];
    st.ux = (R)u[k];
    st.uy = (R)u[ustride + k];
    st.uz = (R)u[2 * ustride + k];
    st.eta = (R)(theta[k] / theta0 - 1.0);
    bool ok = state_ok(st);
    R zero[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) zero[i] = R(0);
    typename Codec::raw_t* out = dst + (int64_t)s * kQ * d.plane + node;
    equilibrium_relax<Codec, EQ>(st, K, R(Codec::kScale), R(0), zero,
                                 [&](auto I, R val) { out[(int64_t)I * d.plane] = Codec::to_raw(val); }, ok);
    if (!ok) atomicOr(err, 1);
}

template <class Codec>
__device__ __forceinline__ NodeMoments<typename Codec::R> node_moments_at(const typename Codec::raw_t* __restrict__ src,
                                                                          const Dims& d, int64_t q,
                                                                          const Consts<typename Codec::R>& K) {
    using R = typename Codec::R;
    const int s = q >= d.plane;
    const int64_t node = q - s * d.plane;
    const typename Codec::raw_t* base = src + (int64_t)s * kQ * d.plane + node;
    R dv[kQ];
    constexpr R inv_scale = R(1.0 / Codec::kScale);
    static_for<kQ>([&](auto I) {
        dv[I] = Codec::dev(Codec::value(base[(int64_t)I * d.plane]), K.w[vel(I).shell] * inv_scale);
    });
    return moments_from_dev(dv);
}

// Moments of nodes q in [q0, q0 + count) into float64 fields indexed by q - q0.
template <class Codec>
__global__ void __launch_bounds__(256) k_moments(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                 Consts<typename Codec::R> K, double theta0, int64_t q0, int64_t count,
                                                 double* __restrict__ rho, double* __restrict__ u, int64_t ustride,
                                                 double* __restrict__ theta) {
    using R = typename Codec::R;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const NodeMoments<R> m = node_moments_at<Codec>(src, d, q0 + k, K);
    const NodeState<R> st = state_from_moments(m, K);
    if (rho) rho[k] = 1.0 + (double)m.drho;
    if (u) {
        u[k] = (double)st.ux;
        u[ustride + k] = (double)st.uy;
        u[2 * ustride + k] = (double)st.uz;
    }
    if (theta) theta[k] = theta0 * (1.0 + (double)st.eta);
}

constexpr int kRedThreads = 256;

// Per-block FP64 partial sums of (drho, jx, jy, jz, dk) over all nodes, in a
// fixed order (grid-stride loop, then a shared-memory tree): deterministic
// for a given grid size.
template <class Codec>
// Over the planes [z0, z0 + nzr) of both sub-lattices (all of them: z0 = 0, nzr = nz).
__global__ void __launch_bounds__(kRedThreads) k_conserved(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                           Consts<typename Codec::R> K, double* __restrict__ partials,
                                                           int64_t z0, int64_t nzr) {
    using R = typename Codec::R;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t nxy = (int64_t)d.nx * d.ny, span = nzr * nxy, n = 2 * span;
    for (int64_t j = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kRedThreads) {
        int64_t q = j;
        if (nzr != d.nz) {
            const int64_t s = j / span;
            q = s * d.plane + z0 * nxy + (j - s * span);
        }
        const NodeMoments<R> m = node_moments_at<Codec>(src, d, q, K);
        acc[0] += (double)m.drho;
        acc[1] += (double)m.jx;
        acc[2] += (double)m.jy;
        acc[3] += (double)m.jz;
        acc[4] += (double)m.dk;
    }
    __shared__ double sh[5][kRedThreads];
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
        for (int k = 0; k < 5; ++k) partials[(int64_t)blockIdx.x * 5 + k] = sh[k][0];
}

// Raw storage <-> float64 populations for elements e in [e0, e0 + count) of the
// [s][41][nz][ny][nx] array; the float64 side is indexed by e - e0.
template <class Codec>
__global__ void __launch_bounds__(256) k_to_f64(const typename Codec::raw_t* __restrict__ src, int64_t plane, W41 w,
                                                int64_t e0, int64_t count, double* __restrict__ f) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int64_t e = e0 + k;
    const int i = (int)((e / plane) % kQ);
    const double v = (double)Codec::value(src[e]);
    if constexpr (Codec::stores_f)
        f[k] = v;
    else
        f[k] = w.w[i] * (1.0 + v * (1.0 / Codec::kScale));
}

template <class Codec>
__global__ void __launch_bounds__(256) k_from_f64(const double* __restrict__ f, int64_t plane, W41 w, int64_t e0,
                                                  int64_t count, typename Codec::raw_t* __restrict__ dst) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int64_t e = e0 + k;
    const int i = (int)((e / plane) % kQ);
    double h;
    if constexpr (Codec::stores_f)
        h = f[k];
    else
        h = (f[k] - w.w[i]) / w.w[i] * Codec::kScale;
    dst[e] = Codec::to_raw((typename Codec::R)h);
}

}  // namespace gblb
