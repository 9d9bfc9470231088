// Isothermal nonideal fluid (Sec. "Nonideal Fluids and two-phase flow"; derivative
// stencil of Appendix A), with the van der Waals, the Peng-Robinson type (Eq. cspreos)
// or the Carnahan-Starling equation of state.
//
// Per step, from the post-collision state src:
//   k_ni_density  rho of the streamed populations, sum_i f_i(x - c_i), and
//                 mu_nid(rho), F_nid(rho) of each node
//   k_ni_fields   per node: grad2 rho (3), lap F_nid and the isotropic part of I_ab,
//                 -(1/2)|grad2 rho|^2 - rho lap rho
//   k_ni_force    g^nid of Eq. (gradientFinal) at the node, from its stencil
//                 neighbours' fields:
//                   rho g = -[rho grad2 mu + mu grad2 rho - eta grad2 F
//                             - (1 - eta) grad4 F + kappa grad2_b I_ab],
//                   grad4 = grad2 - (theta_hat / 2) grad2 lap,
//                   I_ab = [-(1/2)|grad rho|^2 - rho lap rho] delta_ab + grad_a rho grad_b rho
//   k_ni_step     the pull step with the forced BGK collision of
//                 Eq. (multiphaseEvolution), alpha = 2: u = j / rho + g / 2,
//                 f^eq = f^eq(rho, u, theta_0), F_i = g.(c_i - u)/theta_0 f^eq_i,
//                 f' = f + 2 beta (f^eq - f) + (1 - beta) F_i.
// With 16-bit storage and nx even the two gathering passes run on x pairs (k_ni_density2x,
// k_ni_step2x: the x-pair gather of k_step2x, packed FP32x2 arithmetic); with FP32 fields and nx
// even the two stencil passes do too (k_ni_fields2x, k_ni_force2x: the pair's 24 distinct
// neighbours loaded once for both nodes).
// The stencil is the 15-velocity bcc set of Appendix A: rest, (+-1, 0, 0) and
// permutations (on the node's own sub-lattice), (+-1/2, +-1/2, +-1/2) (on the
// other); weights 14/36, 1/36, 2/36; theta_hat = 1/6.  The fields are in
// the storage codec's compute type: FP64 for FP64 storage, FP32 otherwise.
#include <math.h>

#include "lb_ctx.h"
#include "lb_eos.cuh"
#include "lb_kernels.cuh"

namespace gblb {

constexpr double kHatTheta = 1.0 / 6.0;
constexpr int kStencil = 14;  // moving stencil velocities (the rest one only enters lap)

// Doubled velocity and weight of moving stencil velocity k: 6 sc-1 then 8 bcc-1/2.
template <class F>
__device__ __forceinline__ void stencil(int k, int& cx, int& cy, int& cz, F& w) {
    if (k < 6) {
        cx = cy = cz = 0;
        const int v = (k & 1) ? -2 : 2;
        if (k < 2)
            cx = v;
        else if (k < 4)
            cy = v;
        else
            cz = v;
        w = F(1.0 / 36.0);
    } else {
        const int j = k - 6;
        cx = (j & 1) ? -1 : 1;
        cy = (j & 2) ? -1 : 1;
        cz = (j & 4) ? -1 : 1;
        w = F(2.0 / 36.0);
    }
}

constexpr int kNiThreads = 128;

// Field arrays in the compute type F over the n = 2 nx ny nz nodes (field index q, n even).  The
// arrays of two fields hold the nodes in pairs (2p, 2p + 1), p = q >> 1, as four values
// {u(2p), u(2p + 1), v(2p), v(2p + 1)}: an x pair (x even, nx even) reads both nodes' u and v
// in one 16-byte load, and a warp's loads of 32 pairs are contiguous.
//   RF = {rho, F_nid}, MU[q] = mu_nid                              (density pass)
//   A = {mu_nid, F_nid}, B = {lap F_nid, iso}, C = {grad2_x rho, grad2_y rho},
//   D[q] = grad2_z rho                                              (field pass)
//   G[a n + q] = g^nid_a                                            (force pass)
// with iso = -(1/2)|grad2 rho|^2 - rho lap rho, the isotropic part of I_ab.
template <class F>
struct NiFields {
    F* RF;
    F* A;
    F* B;
    F* C;
    F* MU;
    F* D;
    F* G;
};

// Index of u (v = 0) or v (v = 1) of node q in an array of two fields.
__device__ __forceinline__ uint32_t ni_pair_at(uint32_t q, int v) { return 4 * (q >> 1) + 2 * v + (q & 1); }

// Four values of one pair in the field type (the 16-byte load of a pair with F = float).
template <class F>
struct alignas(4 * sizeof(F)) NiQuad {
    F x, y, z, w;
};
// u (v = 0) or v (v = 1) of the pair's node c.
template <class F>
__device__ __forceinline__ F quad_at(const NiQuad<F>& r, int v, int c) {
    return v ? (c ? r.w : r.z) : (c ? r.y : r.x);
}

// a in [0, n] (wrap_up) or in [-1, n) (wrap_dn) back into [0, n): the stencil's offsets are +-1.
__device__ __forceinline__ uint32_t wrap_up(int a, int n) { return (uint32_t)(a == n ? 0 : a); }
__device__ __forceinline__ uint32_t wrap_dn(int a, int n) { return (uint32_t)(a < 0 ? n - 1 : a); }

// Node of this thread: blocks cover (row, x chunk) pairs, rows running (z, s, y) with y fastest, so
// that the two sub-lattices of a plane are visited together (the stencil passes read the other
// sub-lattice's fields, which then come from L2).  The coordinates come from 32-bit divisions of
// the block index (2 ny nz < 2^31, checked at init); q is the node's field index
// ((s nz + z) ny + y) nx + x.
__device__ __forceinline__ bool ni_node(const Dims& d, int chunks, int64_t& q, int& s, int& z, int& y, int& x) {
    const uint32_t b = blockIdx.x;
    const uint32_t row = b / (uint32_t)chunks;
    x = (int)(b - row * (uint32_t)chunks) * kNiThreads + (int)threadIdx.x;
    if (x >= d.nx) return false;
    const uint32_t zs = row / (uint32_t)d.ny;
    y = (int)(row - zs * (uint32_t)d.ny);
    z = (int)(zs >> 1);
    s = (int)(zs & 1u);
    q = (((int64_t)s * d.nz + z) * d.ny + y) * d.nx + x;
    return true;
}

// Field indices of the 14 moving stencil neighbours of node (s, z, y, x), in the order of
// stencil(): the sc-1 links +x, -x, +y, -y, +z, -z on the node's own sub-lattice, then the
// bcc-1/2 links on the other, whose +1/2 neighbour along an axis has index coordinate + s and
// whose -1/2 neighbour has + s - 1.  32-bit: 2 nx ny nz < 2^32 (checked when the mode is enabled).
__device__ __forceinline__ void ni_neighbors(const Dims& d, int s, int z, int y, int x, uint32_t (&m)[kStencil]) {
    const uint32_t nx = (uint32_t)d.nx, nxy = nx * (uint32_t)d.ny, pl = (uint32_t)d.plane;
    const uint32_t own = (uint32_t)s * pl, oth = (uint32_t)(1 - s) * pl;
    const uint32_t xs = (uint32_t)x, ys = (uint32_t)y * nx, zs = (uint32_t)z * nxy;
    m[0] = own + zs + ys + wrap_up(x + 1, d.nx);
    m[1] = own + zs + ys + wrap_dn(x - 1, d.nx);
    m[2] = own + zs + wrap_up(y + 1, d.ny) * nx + xs;
    m[3] = own + zs + wrap_dn(y - 1, d.ny) * nx + xs;
    m[4] = own + wrap_up(z + 1, d.nz) * nxy + ys + xs;
    m[5] = own + wrap_dn(z - 1, d.nz) * nxy + ys + xs;
    const uint32_t X[2] = {wrap_up(x + s, d.nx), wrap_dn(x + s - 1, d.nx)};
    const uint32_t Y[2] = {wrap_up(y + s, d.ny) * nx, wrap_dn(y + s - 1, d.ny) * nx};
    const uint32_t Z[2] = {wrap_up(z + s, d.nz) * nxy, wrap_dn(z + s - 1, d.nz) * nxy};
#pragma unroll
    for (int j = 0; j < 8; ++j) m[6 + j] = oth + Z[(j >> 2) & 1] + Y[(j >> 1) & 1] + X[j & 1];
}

// The pull gather of step_node: v[i] = f_i(x - c_i) in the codec's working value.
template <class Codec>
__device__ __forceinline__ void ni_gather(const typename Codec::raw_t* __restrict__ src, const Dims& d, int s, int z,
                                          int y, int x, typename Codec::R (&v)[kQ]) {
    using T = typename Codec::raw_t;
    const int64_t nxy = (int64_t)d.nx * d.ny;
    int xs[5];
    int64_t yo[5], zo[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        xs[k] = wrap(x - (k - 2), d.nx);
        yo[k] = (int64_t)wrap(y - (k - 2), d.ny) * d.nx;
        zo[k] = (int64_t)wrap(z - (k - 2), d.nz) * nxy;
    }
    const int hxp = s ? xs[2] : xs[3], hxm = s ? xs[1] : xs[2];
    const int64_t hyp = s ? yo[2] : yo[3], hym = s ? yo[1] : yo[2];
    const int64_t hzp = s ? zo[2] : zo[3], hzm = s ? zo[1] : zo[2];
    const T* same = src + (int64_t)s * kQ * d.plane;
    const T* other = src + (int64_t)(1 - s) * kQ * d.plane;
    static_for<kQ>([&](auto I) {
        constexpr Vel c = vel(I);
        if constexpr (c.shell == 5) {
            const int64_t off = (c.z > 0 ? hzp : hzm) + (c.y > 0 ? hyp : hym) + (c.x > 0 ? hxp : hxm);
            v[I] = Codec::value(other[(int64_t)I * d.plane + off]);
        } else {
            const int64_t off = zo[c.z / 2 + 2] + yo[c.y / 2 + 2] + xs[c.x / 2 + 2];
            v[I] = Codec::value(same[(int64_t)I * d.plane + off]);
        }
    });
}

template <class Codec>
__global__ void __launch_bounds__(kNiThreads) k_ni_density(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                           int chunks, Consts<typename Codec::R> K, NiEosT<typename Codec::R> e,
                                                           NiFields<typename Codec::R> fl) {
    using R = typename Codec::R;
    int64_t q;
    int s, z, y, x;
    if (!ni_node(d, chunks, q, s, z, y, x)) return;
    R v[kQ];
    ni_gather<Codec>(src, d, s, z, y, x, v);
    R dr = 0;  // rho - 1 = sum_i (f_i - w_i)
    static_for<kQ>([&](auto I) { dr += Codec::dev(v[I], K.w[vel(I).shell] * R(1.0 / Codec::kScale)); });
    const R r = R(1) + dr;
    R mu, Fe;
    ni_eos<R>(r, e, mu, Fe);
    const uint32_t qq = (uint32_t)q;
    fl.RF[ni_pair_at(qq, 0)] = r;
    fl.RF[ni_pair_at(qq, 1)] = Fe;
    fl.MU[qq] = mu;
}

// Every moving stencil term of a first derivative carries w_k c_ka / 2 = +-1/36 (sc-1: 1/36 x +-1,
// bcc-1/2: 2/36 x +-1/2), so the passes sum the neighbours' values with signs and apply the weight
// once; grad2 X = (1 / (36 theta_hat)) sum_k sgn(c_ka) X(x + c_k) over the k with c_ka != 0.
constexpr double kGradScale = 1.0 / (36.0 * kHatTheta);

// acc += v for sign > 0, acc -= v otherwise (the sign is a compile-time constant after unrolling).
template <class F>
__device__ __forceinline__ void add_signed(F& acc, F v, int sign) {
    acc = sign > 0 ? acc + v : acc - v;
}

// The field pass at one node from its rho0, F0 and its neighbours' rn, Fn (in the order of
// stencil()): grad2 rho, lap F_nid and iso.  The Laplacian sums the neighbours' differences from
// the node, lap X = (2 / theta_hat) sum_k w_k (X(x + c_k) - X(x)) = (1/3) [sum_sc dX + 2 sum_bcc
// dX], each difference formed before it is added (close values subtract exactly).
template <class F>
__device__ __forceinline__ void ni_fields_node(F r0, F F0, const F (&rn)[kStencil], const F (&Fn)[kStencil],
                                               F (&g)[3], F& lapF, F& iso) {
    F gsum[3] = {F(0), F(0), F(0)}, lr[2] = {F(0), F(0)}, lF[2] = {F(0), F(0)};
#pragma unroll
    for (int k = 0; k < kStencil; ++k) {
        int cx, cy, cz;
        F w;
        stencil(k, cx, cy, cz, w);
        if (cx) add_signed(gsum[0], rn[k], cx);
        if (cy) add_signed(gsum[1], rn[k], cy);
        if (cz) add_signed(gsum[2], rn[k], cz);
        const int sh = k < 6 ? 0 : 1;  // sc-1 or bcc-1/2
        lr[sh] += rn[k] - r0;
        lF[sh] += Fn[k] - F0;
    }
    const F gs = F(kGradScale);
    for (int b = 0; b < 3; ++b) g[b] = gsum[b] * gs;
    const F lap = F(1.0 / 3.0) * (lr[0] + F(2) * lr[1]);
    iso = F(-0.5) * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) - r0 * lap;
    lapF = F(1.0 / 3.0) * (lF[0] + F(2) * lF[1]);
}

template <class F>
__global__ void __launch_bounds__(kNiThreads) k_ni_fields(Dims d, int chunks, NiFields<F> fl) {
    int64_t q64;
    int s, z, y, x;
    if (!ni_node(d, chunks, q64, s, z, y, x)) return;
    const uint32_t q = (uint32_t)q64;
    uint32_t nb[kStencil];
    ni_neighbors(d, s, z, y, x, nb);
    F rn[kStencil], Fn[kStencil];
#pragma unroll
    for (int k = 0; k < kStencil; ++k) {
        rn[k] = fl.RF[ni_pair_at(nb[k], 0)];
        Fn[k] = fl.RF[ni_pair_at(nb[k], 1)];
    }
    const F F0 = fl.RF[ni_pair_at(q, 1)];
    F g[3], lapF, iso;
    ni_fields_node<F>(fl.RF[ni_pair_at(q, 0)], F0, rn, Fn, g, lapF, iso);
    fl.A[ni_pair_at(q, 0)] = fl.MU[q];
    fl.A[ni_pair_at(q, 1)] = F0;
    fl.B[ni_pair_at(q, 0)] = lapF;
    fl.B[ni_pair_at(q, 1)] = iso;
    fl.C[ni_pair_at(q, 0)] = g[0];
    fl.C[ni_pair_at(q, 1)] = g[1];
    fl.D[q] = g[2];
}

// A stencil neighbour's fields as the force pass uses them.
template <class F>
struct NiNb {
    F mu, Fe, lF, iso, g[3];
};

// One stencil neighbour's terms of the force sums, k its stencil velocity (doubled c: sc-1 +-2
// along one axis; bcc-1/2 +-1 along each).  With sgn(c_a) = c_a / |c_a|:
//   dmu_a, dF_a, dlF_a += sgn(c_a) mu, F, lap F                                  (c_a != 0)
//   divI_a += sum_b sgn(c_b) I_ab = grad_a rho sum_b sgn(c_b) grad_b rho + sgn(c_a) iso;
// each sum times 1 / (36 theta_hat) is the grad2 of Appendix A.
template <class F>
struct NiForceSums {
    F dmu[3], dF[3], dlF[3], divI[3];
};
template <class F>
__device__ __forceinline__ void ni_sums_zero(NiForceSums<F>& a) {
    for (int b = 0; b < 3; ++b) a.dmu[b] = a.dF[b] = a.dlF[b] = a.divI[b] = F(0);
}
template <class F>
__device__ __forceinline__ void ni_force_term(NiForceSums<F>& a, int k, const NiNb<F>& v) {
    int cc[3];
    F w;
    stencil(k, cc[0], cc[1], cc[2], w);
    F cg = F(0);  // sum_b sgn(c_b) grad_b rho
    bool first = true;
    for (int b = 0; b < 3; ++b) {
        if (cc[b] == 0) continue;
        add_signed(a.dmu[b], v.mu, cc[b]);
        add_signed(a.dF[b], v.Fe, cc[b]);
        add_signed(a.dlF[b], v.lF, cc[b]);
        if (first)
            cg = cc[b] > 0 ? v.g[b] : -v.g[b];
        else
            add_signed(cg, v.g[b], cc[b]);
        first = false;
    }
    for (int b = 0; b < 3; ++b) {
        a.divI[b] = fma(v.g[b], cg, a.divI[b]);
        if (cc[b]) add_signed(a.divI[b], v.iso, cc[b]);
    }
}

// g^nid from the sums and the node's own rho, mu and grad2 rho:
//   rho g = -[rho grad2 mu + mu grad2 rho - eta grad2 F - (1 - eta) grad4 F + kappa grad2_b I_ab].
template <class F>
__device__ __forceinline__ void ni_force_finish(const NiEosT<F>& e, const NiForceSums<F>& a, F r0, F mu0,
                                                const F (&g2r)[3], F (&g)[3]) {
    const F gs = F(kGradScale), inv_r0 = F(1) / r0;
    for (int b = 0; b < 3; ++b) {
        const F g2mu = a.dmu[b] * gs, g2F = a.dF[b] * gs, g2lF = a.dlF[b] * gs;
        const F g4F = g2F - F(0.5 * kHatTheta) * g2lF;
        const F rg = -(r0 * g2mu + mu0 * g2r[b] - e.eta * g2F - (F(1) - e.eta) * g4F + e.kappa * a.divI[b] * gs);
        g[b] = rg * inv_r0;
    }
}

// g^nid of every node into G (a pass of its own: folded into the step, the stencil sums raise the
// step's register count and the fused step ran slower than the two passes).
template <class F>
__global__ void __launch_bounds__(kNiThreads) k_ni_force(Dims d, int chunks, NiEosT<F> e, NiFields<F> fl) {
    int64_t q64;
    int s, z, y, x;
    if (!ni_node(d, chunks, q64, s, z, y, x)) return;
    const uint32_t q = (uint32_t)q64;
    uint32_t nb[kStencil];
    ni_neighbors(d, s, z, y, x, nb);
    NiForceSums<F> a;
    ni_sums_zero(a);
#pragma unroll
    for (int k = 0; k < kStencil; ++k) {
        const uint32_t m = nb[k];
        const NiNb<F> v{fl.A[ni_pair_at(m, 0)], fl.A[ni_pair_at(m, 1)], fl.B[ni_pair_at(m, 0)],
                        fl.B[ni_pair_at(m, 1)], {fl.C[ni_pair_at(m, 0)], fl.C[ni_pair_at(m, 1)], fl.D[m]}};
        ni_force_term<F>(a, k, v);
    }
    const F g2r[3] = {fl.C[ni_pair_at(q, 0)], fl.C[ni_pair_at(q, 1)], fl.D[q]};
    F g[3];
    ni_force_finish<F>(e, a, fl.RF[ni_pair_at(q, 0)], fl.A[ni_pair_at(q, 0)], g2r, g);
    const size_t n = 2 * (size_t)d.plane;
    for (int b = 0; b < 3; ++b) fl.G[b * n + q] = g[b];
}

// Two x-adjacent nodes (x even, nx even) per thread in the stencil passes, rows in the (z, s, y)
// order of ni_node; q is the even node's field index, q >> 1 the pair's.
__device__ __forceinline__ bool ni_pair_zsy(const Dims& d, int chunks, uint32_t& q, int& s, int& z, int& y, int& x) {
    const uint32_t b = blockIdx.x;
    const uint32_t row = b / (uint32_t)chunks;
    x = 2 * ((int)(b - row * (uint32_t)chunks) * (int)blockDim.x + (int)threadIdx.x);
    if (x >= d.nx) return false;
    const uint32_t zs = row / (uint32_t)d.ny;
    y = (int)(row - zs * (uint32_t)d.ny);
    z = (int)(zs >> 1);
    s = (int)(zs & 1u);
    q = (((uint32_t)s * (uint32_t)d.nz + (uint32_t)z) * (uint32_t)d.ny + (uint32_t)y) * (uint32_t)d.nx + (uint32_t)x;
    return true;
}

// The stencil neighbours of the pair (x, x + 1) on sub-lattice S lie in 15 pairs (pair indices):
//   0-2    the own row's pairs at x - 2, x, x + 2 (wrapped)
//   3-6    the rows +y, -y, +z, -z at x
//   7-10   the other sub-lattice's rows c = 0..3 of the bcc-1/2 links at x (y side c & 1, z side
//          c >> 1; side 0 is the +1/2 one)
//   11-14  the same rows at x - 2 (S = 0) or x + 2 (S = 1)
constexpr int kPairPos = 15;
template <int S>
__device__ __forceinline__ void ni_pair_positions(const Dims& d, int z, int y, int x, uint32_t q,
                                                  uint32_t (&p)[kPairPos]) {
    const uint32_t nx = (uint32_t)d.nx, nxy = nx * (uint32_t)d.ny, pl = (uint32_t)d.plane;
    const uint32_t own = (uint32_t)S * pl, oth = (uint32_t)(1 - S) * pl, hx = nx / 2;
    const uint32_t xs = (uint32_t)x, ys = (uint32_t)y * nx, zs = (uint32_t)z * nxy;
    const bool first = x == 0, last = x + 2 == d.nx;
    auto left = [&](uint32_t r) { return first ? r + hx - 1 : r - 1; };   // the pair at x - 2 of r's row
    auto right = [&](uint32_t r) { return last ? r + 1 - hx : r + 1; };  // the pair at x + 2
    const uint32_t pq = q >> 1;
    p[0] = left(pq);
    p[1] = pq;
    p[2] = right(pq);
    p[3] = (own + zs + wrap_up(y + 1, d.ny) * nx + xs) >> 1;
    p[4] = (own + zs + wrap_dn(y - 1, d.ny) * nx + xs) >> 1;
    p[5] = (own + wrap_up(z + 1, d.nz) * nxy + ys + xs) >> 1;
    p[6] = (own + wrap_dn(z - 1, d.nz) * nxy + ys + xs) >> 1;
    const uint32_t Y[2] = {wrap_up(y + S, d.ny) * nx, wrap_dn(y + S - 1, d.ny) * nx};
    const uint32_t Z[2] = {wrap_up(z + S, d.nz) * nxy, wrap_dn(z + S - 1, d.nz) * nxy};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        p[7 + c] = (oth + Z[c >> 1] + Y[c & 1] + xs) >> 1;
        p[11 + c] = S ? right(p[7 + c]) : left(p[7 + c]);
    }
}

// 2 x (pair position) + node within it of stencil neighbour k of node x + h.
template <int S>
__host__ __device__ constexpr int ni_pair_src(int h, int k) {
    if (k == 0) return h ? 2 * 2 + 0 : 2 * 1 + 1;  // +x: x + 1, x + 2
    if (k == 1) return h ? 2 * 1 + 0 : 2 * 0 + 1;  // -x: x - 1, x
    if (k < 6) return 2 * (k + 1) + h;             // +-y, +-z: the same x
    const int c = (k - 6) >> 1;
    const int o = ((k - 6) & 1) ? S - 1 + h : S + h;  // x offset of the bcc-1/2 neighbour
    return o < 0 ? 2 * (11 + c) + 1 : o == 0 ? 2 * (7 + c) : o == 1 ? 2 * (7 + c) + 1 : 2 * (11 + c);
}

template <class F>
struct alignas(2 * sizeof(F)) NiDuo {
    F x, y;
};

template <class F, int S>
__device__ __forceinline__ void ni_fields_pair(const Dims& d, const NiFields<F>& fl, int z, int y, int x, uint32_t q) {
    uint32_t p[kPairPos];
    ni_pair_positions<S>(d, z, y, x, q, p);
    const NiQuad<F>* RF = reinterpret_cast<const NiQuad<F>*>(fl.RF);
    NiQuad<F> rf[kPairPos];
#pragma unroll
    for (int i = 0; i < kPairPos; ++i) rf[i] = RF[p[i]];
    const NiDuo<F> mu = *reinterpret_cast<const NiDuo<F>*>(fl.MU + q);
    F g[2][3], lapF[2], iso[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        F rn[kStencil], Fn[kStencil];
#pragma unroll
        for (int k = 0; k < kStencil; ++k) {
            const int src = ni_pair_src<S>(h, k);
            rn[k] = quad_at(rf[src >> 1], 0, src & 1);
            Fn[k] = quad_at(rf[src >> 1], 1, src & 1);
        }
        ni_fields_node<F>(quad_at(rf[1], 0, h), quad_at(rf[1], 1, h), rn, Fn, g[h], lapF[h], iso[h]);
    }
    const uint32_t pq = q >> 1;
    reinterpret_cast<NiQuad<F>*>(fl.A)[pq] = NiQuad<F>{mu.x, mu.y, rf[1].z, rf[1].w};
    reinterpret_cast<NiQuad<F>*>(fl.B)[pq] = NiQuad<F>{lapF[0], lapF[1], iso[0], iso[1]};
    reinterpret_cast<NiQuad<F>*>(fl.C)[pq] = NiQuad<F>{g[0][0], g[1][0], g[0][1], g[1][1]};
    *reinterpret_cast<NiDuo<F>*>(fl.D + q) = NiDuo<F>{g[0][2], g[1][2]};
}

// k_ni_fields for an x pair.
template <class F>
__global__ void __launch_bounds__(kNiThreads) k_ni_fields2x(Dims d, int chunks, NiFields<F> fl) {
    uint32_t q;
    int s, z, y, x;
    if (!ni_pair_zsy(d, chunks, q, s, z, y, x)) return;
    if (s)
        ni_fields_pair<F, 1>(d, fl, z, y, x, q);
    else
        ni_fields_pair<F, 0>(d, fl, z, y, x, q);
}

template <class F, int S>
__device__ __forceinline__ void ni_force_pair(const Dims& d, const NiEosT<F>& e, const NiFields<F>& fl, int z, int y,
                                              int x, uint32_t q) {
    uint32_t p[kPairPos];
    ni_pair_positions<S>(d, z, y, x, q, p);
    const NiQuad<F>* A = reinterpret_cast<const NiQuad<F>*>(fl.A);
    const NiQuad<F>* B = reinterpret_cast<const NiQuad<F>*>(fl.B);
    const NiQuad<F>* C = reinterpret_cast<const NiQuad<F>*>(fl.C);
    const NiDuo<F>* D = reinterpret_cast<const NiDuo<F>*>(fl.D);
    NiQuad<F> qa[kPairPos], qb[kPairPos], qc[kPairPos];
    NiDuo<F> qd[kPairPos];
#pragma unroll
    for (int i = 0; i < kPairPos; ++i) {
        qa[i] = A[p[i]];
        qb[i] = B[p[i]];
        qc[i] = C[p[i]];
        qd[i] = D[p[i]];
    }
    NiForceSums<F> a[2];
    ni_sums_zero(a[0]);
    ni_sums_zero(a[1]);
#pragma unroll
    for (int k = 0; k < kStencil; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int src = ni_pair_src<S>(h, k), i = src >> 1, c = src & 1;
            const NiNb<F> v{quad_at(qa[i], 0, c), quad_at(qa[i], 1, c), quad_at(qb[i], 0, c), quad_at(qb[i], 1, c),
                            {quad_at(qc[i], 0, c), quad_at(qc[i], 1, c), c ? qd[i].y : qd[i].x}};
            ni_force_term<F>(a[h], k, v);
        }
    }
    const NiQuad<F> rf = reinterpret_cast<const NiQuad<F>*>(fl.RF)[q >> 1];
    F g[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const F g2r[3] = {quad_at(qc[1], 0, h), quad_at(qc[1], 1, h), h ? qd[1].y : qd[1].x};
        ni_force_finish<F>(e, a[h], quad_at(rf, 0, h), quad_at(qa[1], 0, h), g2r, g[h]);
    }
    const size_t n = 2 * (size_t)d.plane;
    for (int b = 0; b < 3; ++b) *reinterpret_cast<NiDuo<F>*>(fl.G + b * n + q) = NiDuo<F>{g[0][b], g[1][b]};
}

// k_ni_force for an x pair.  80 registers (6 blocks per SM), without spills: 2.86 against 2.92 ms
// for the 256^3 step at 128 registers (4 blocks).
template <class F>
__global__ void __launch_bounds__(kNiThreads, 6) k_ni_force2x(Dims d, int chunks, NiEosT<F> e, NiFields<F> fl) {
    uint32_t q;
    int s, z, y, x;
    if (!ni_pair_zsy(d, chunks, q, s, z, y, x)) return;
    if (s)
        ni_force_pair<F, 1>(d, e, fl, z, y, x, q);
    else
        ni_force_pair<F, 0>(d, e, fl, z, y, x, q);
}

// The pull step with the forced BGK collision; g^nid from G.
template <class Codec>
__global__ void __launch_bounds__(kNiThreads) k_ni_step(const typename Codec::raw_t* __restrict__ src,
                                                        typename Codec::raw_t* __restrict__ dst, Dims d, int chunks,
                                                        Consts<typename Codec::R> K, typename Codec::R tb,
                                                        typename Codec::R inv_theta0,
                                                        const typename Codec::R* __restrict__ G,
                                                        int* __restrict__ err) {
    using R = typename Codec::R;
    using T = typename Codec::raw_t;
    int64_t q;
    int s, z, y, x;
    if (!ni_node(d, chunks, q, s, z, y, x)) return;
    const int64_t n = 2 * d.plane;
    const R gf[3] = {G[q], G[n + q], G[2 * n + q]};
    R v[kQ];
    ni_gather<Codec>(src, d, s, z, y, x, v);
    R dv[kQ];
    constexpr R inv_scale = R(1.0 / Codec::kScale);
    static_for<kQ>([&](auto I) { dv[I] = Codec::dev(v[I], K.w[vel(I).shell] * inv_scale); });
    const NodeMoments<R> m = moments_from_dev(dv);
    NodeState<R> st;
    st.drho = m.drho;
    st.rho = R(1) + m.drho;
    const R gx = gf[0], gy = gf[1], gz = gf[2];
    const R inv_rho = R(1) / st.rho;
    st.ux = m.jx * inv_rho + R(0.5) * gx;
    st.uy = m.jy * inv_rho + R(0.5) * gy;
    st.uz = m.jz * inv_rho + R(0.5) * gz;
    st.eta = R(0);  // isothermal: the equilibrium at theta_0
    bool ok = state_ok(st);
    // f^eq in the working representation: f (FP64 codec) or scale * h^eq (deviation codecs)
    R veq[kQ], zero[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) zero[i] = R(0);
    equilibrium_relax<Codec, 1>(st, K, R(Codec::kScale), R(0), zero, [&](auto I, R val) { veq[I] = val; }, ok);
    T* out = dst + (int64_t)s * kQ * d.plane + ((int64_t)z * d.ny + y) * d.nx + x;
    const R half_f = R(1) - R(0.5) * tb;  // 1 - beta
    static_for<kQ>([&](auto I) {
        constexpr Vel c = vel(I);
        const R gc = gx * (R(0.5 * c.x) - st.ux) + gy * (R(0.5 * c.y) - st.uy) + gz * (R(0.5 * c.z) - st.uz);
        R val;
        if constexpr (Codec::stores_f) {
            const R F = gc * inv_theta0 * veq[I];
            val = v[I] + tb * (veq[I] - v[I]) + half_f * F;
        } else {
            // F_i / w_i = gc / theta0 (1 + h^eq), in units of the stored scale
            const R F = gc * inv_theta0 * (R(Codec::kScale) + veq[I]);
            val = v[I] + tb * (veq[I] - v[I]) + half_f * F;
        }
        out[(int64_t)I * d.plane] = Codec::to_raw(val);
    });
    if (!ok) atomicOr(err, 1);
}

// Two x-adjacent nodes per thread (16-bit storage, nx even): the x-pair gather of k_step2x and
// packed FP32x2 arithmetic; x is the thread's even node.  ni_pair: one row per block, blocks over
// (row, chunk of x pairs), rows (s, z, y); q the field index of the even node.
__device__ __forceinline__ bool ni_pair(const Dims& d, int chunks, uint32_t& q, int& s, int& z, int& y, int& x) {
    const uint32_t b = blockIdx.x;
    const uint32_t row = b / (uint32_t)chunks;
    x = 2 * ((int)(b - row * (uint32_t)chunks) * (int)blockDim.x + (int)threadIdx.x);
    if (x >= d.nx) return false;
    const uint32_t zr = row / (uint32_t)d.ny;
    y = (int)(row - zr * (uint32_t)d.ny);
    s = (int)(zr / (uint32_t)d.nz);
    z = (int)(zr - (uint32_t)s * (uint32_t)d.nz);
    q = row * (uint32_t)d.nx + (uint32_t)x;
    return true;
}

template <class Codec>
__device__ __forceinline__ void ni_gather2x(const typename Codec::raw_t* __restrict__ src, const Dims& d, int s, int z,
                                            int y, int x, typename Codec::pair_t (&pv)[kQ]) {
    const uint32_t xm = (uint32_t)wrap(x - 2, d.nx), x0 = (uint32_t)x, xq = (uint32_t)wrap(x + 2, d.nx);
    RowAddr2x<Codec> a;
    a.set(src, d, s, z, y);
    static_for<kQ>([&](auto I) { pv[I] = load_pair2x<Codec, I>(a, (uint32_t)d.plane, xm, x0, xq); });
}

// The rows of a block of the x-pair forced step: `rpb` consecutive rows (s, z, y) for one chunk
// of x pairs, as in the energy-conserving x-pair kernel's L2 mode.  At the start of a row, threads
// 0..40 each prefetch into L2 the next row's source row of their population, and threads 41 ..
// call extra(j = thread - 41, next row, xa, xb) for other spans to prefetch; body(q, s, z, y, x)
// then does the thread's pair of the row (q its field index, x even).
template <class Codec, class Extra, class Body>
__device__ __forceinline__ void ni_row_walk(const typename Codec::raw_t* __restrict__ src, const Dims& d, int chunks,
                                            int rpb, Extra extra, Body body) {
    const uint32_t grp = blockIdx.x / (uint32_t)chunks;
    const int chunk = (int)(blockIdx.x - grp * (uint32_t)chunks);
    const int x = 2 * (chunk * (int)blockDim.x + (int)threadIdx.x);
    const int xa = 2 * chunk * (int)blockDim.x, xb = min(xa + 2 * (int)blockDim.x, d.nx);
    const uint32_t r0 = grp * (uint32_t)rpb, r1 = min(r0 + (uint32_t)rpb, (uint32_t)d.rows);
    int y = (int)(r0 % (uint32_t)d.ny);
    const uint32_t zr = r0 / (uint32_t)d.ny;
    int z = (int)(zr % (uint32_t)d.nz), s = (int)(zr / (uint32_t)d.nz);
    const bool active = x < d.nx;
    for (uint32_t r = r0; r < r1; ++r) {
        int yn = y + 1, zn = z, sn = s;
        if (yn == d.ny) {
            yn = 0;
            if (++zn == d.nz) {
                zn = 0;
                ++sn;
            }
        }
        if (r + 1 < r1) {
            if (threadIdx.x < kQ)
                prefetch_row_l2<Codec>(src, d, (int)threadIdx.x, sn, zn, yn, xa, xb);
            else
                extra((int)threadIdx.x - kQ, r + 1, xa, xb);
        }
        if (active) body(r * (uint32_t)d.nx + (uint32_t)x, s, z, y, x);
        s = sn;
        z = zn;
        y = yn;
    }
}

// L2 prefetch of the whole 16-byte units inside [p0, p1).
__device__ __forceinline__ void prefetch_span_l2(const void* p0, const void* p1) {
    const uintptr_t b0 = ((uintptr_t)p0 + 15) & ~(uintptr_t)15, b1 = (uintptr_t)p1 & ~(uintptr_t)15;
    if (b1 > b0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"((uint32_t)(b1 - b0)) : "memory");
}

// k_ni_density for an x pair (one row per block: the L2 prefetch of the next row, which helps the
// step, measured slower here, 0.617 against 0.538 ms at 256^3).
template <class Codec>
__global__ void __launch_bounds__(kStepThreads) k_ni_density2x(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                               int chunks, Consts<float> K, NiEosT<float> e,
                                                               NiFields<float> fl) {
    uint32_t q;
    int s, z, y, x;
    if (!ni_pair(d, chunks, q, s, z, y, x)) return;
    typename Codec::pair_t pv[kQ];
    ni_gather2x<Codec>(src, d, s, z, y, x, pv);
    constexpr float inv_scale = (float)(1.0 / Codec::kScale);
    F2 dr(0.f);  // rho - 1 = sum_i (f_i - w_i), in the population order of k_ni_density
    static_for<kQ>([&](auto I) { dr += F2(Codec::unpack2(pv[I])) * F2(K.w[vel(I).shell] * inv_scale); });
    const F2 r = F2(1.f) + dr;
    float mu0, F0, mu1, F1;
    ni_eos<float>(r.v.x, e, mu0, F0);
    ni_eos<float>(r.v.y, e, mu1, F1);
    *reinterpret_cast<float4*>(fl.RF + 2 * q) = make_float4(r.v.x, r.v.y, F0, F1);
    *reinterpret_cast<float2*>(fl.MU + q) = make_float2(mu0, mu1);
}

// k_ni_step for an x pair: the forcing is applied as each population's equilibrium is formed.
template <class Codec>
__global__ void __launch_bounds__(kStepThreads, 3) k_ni_step2x(const typename Codec::raw_t* __restrict__ src,
                                                               typename Codec::raw_t* __restrict__ dst, Dims d,
                                                               int chunks, int rpb, Consts<float> K, float tb,
                                                               float inv_theta0, const float* __restrict__ G,
                                                               int* __restrict__ err) {
    using P = typename Codec::pair_t;
    using C2 = Codec2<Codec>;
    const size_t n = 2 * (size_t)d.plane;
    // threads 41..43 prefetch the next row's span of g_x, g_y, g_z
    auto g_rows = [&](int j, uint32_t row, int xa, int xb) {
        if (j < 3) {
            const float* g = G + (size_t)j * n + (size_t)row * (uint32_t)d.nx;
            prefetch_span_l2(g + xa, g + xb);
        }
    };
    ni_row_walk<Codec>(src, d, chunks, rpb, g_rows, [&](uint32_t q, int s, int z, int y, int x) {
    P pv[kQ];
    ni_gather2x<Codec>(src, d, s, z, y, x, pv);
    auto vget = [&](auto I) { return F2(Codec::unpack2(pv[I])); };
    const F2 gx(*reinterpret_cast<const float2*>(G + q)), gy(*reinterpret_cast<const float2*>(G + n + q)),
        gz(*reinterpret_cast<const float2*>(G + 2 * n + q));
    constexpr float inv_scale = (float)(1.0 / Codec::kScale);
    const NodeMoments<F2> m =
        moments_from<F2>([&](auto I) { return C2::dev(vget(I), F2(K.w[vel(I).shell] * inv_scale)); });
    NodeState<F2> st;
    st.drho = m.drho;
    st.rho = F2(1.f) + m.drho;
    const F2 inv_rho = recip(st.rho);
    st.ux = fma(F2(0.5f), gx, m.jx * inv_rho);
    st.uy = fma(F2(0.5f), gy, m.jy * inv_rho);
    st.uz = fma(F2(0.5f), gz, m.jz * inv_rho);
    st.eta = F2(0.f);  // isothermal: the equilibrium at theta_0
    if (!state_ok(st)) atomicOr(err, 1);
    // F_i / w_i = g.(c_i - u) / theta0 (1 + h^eq_i), in units of the stored scale
    const F2 it(inv_theta0);
    const F2 hx = gx * it, hy = gy * it, hz = gz * it;
    const F2 hu = hx * st.ux + hy * st.uy + hz * st.uz;
    const F2 tbv(tb), half_f(1.f - 0.5f * tb), scale((float)Codec::kScale);
    P* outp = reinterpret_cast<P*>(dst + (size_t)s * kQ * d.plane + (q - (uint32_t)s * (uint32_t)d.plane));
    const size_t pstride = (size_t)d.plane / 2;
    equilibrium_relax_g<C2, true>(st, K, scale, F2(0.f), vget, [&](auto I, F2 veq) {
        constexpr Vel c = vel(I);
        F2 gc = F2(0.f) - hu;
        if constexpr (c.x != 0) gc = fma(F2(0.5f * c.x), hx, gc);
        if constexpr (c.y != 0) gc = fma(F2(0.5f * c.y), hy, gc);
        if constexpr (c.z != 0) gc = fma(F2(0.5f * c.z), hz, gc);
        const F2 v = vget(I);
        const F2 val = fma(half_f, gc * (scale + veq), fma(tbv, veq - v, v));
        outp[(size_t)I * pstride] = Codec::to_raw2(val.v);
    });
    });
}

template <class F>
static cudaError_t ni_codec(int prec, F&& f) {
    switch (prec) {
        case kF64: return f(CodecF64{});
        case kF32: return f(CodecF32{});
        case kF16: return f(CodecF16{});
        case kBF16: return f(CodecBF16{});
        default: return cudaErrorInvalidValue;
    }
}

// The field arrays RF, A, B, C (2 values per node each), MU, D (1) and G (3), in the field type.
size_t nonideal_doubles(const Dims& d, int prec) {
    const size_t values = (size_t)13 * 2 * d.plane;
    return prec == kF64 ? values : (values + 1) / 2;
}

cudaError_t launch_nonideal_step(int prec, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                                 double twobeta, int kind, const double eos[4], double* work, int* err,
                                 cudaStream_t st) {
    const int64_t n = 2 * d.plane;
    const int chunks = (d.nx + kNiThreads - 1) / kNiThreads;
    const unsigned blocks = (unsigned)(d.rows * chunks);
    if (kind < kVdW || kind > kCarnahanStarling) return cudaErrorInvalidValue;
    const NiEos e64{eos[0], eos[1], c.theta0, eos[2], eos[3], kind};
    return ni_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        using R = typename C::R;
        const Consts<R>* K;
        if constexpr (sizeof(R) == 8)
            K = &c.kd;
        else
            K = &c.kf;
        const NiEosT<R> e = ni_eos_in<R>(e64);
        // field arrays in the compute type: RF, A, B, C (2 values per node each; 16-byte aligned, n
        // is even), then MU, D (1) and G (3)
        NiFields<R> fl;
        fl.RF = reinterpret_cast<R*>(work);
        fl.A = fl.RF + 2 * n;
        fl.B = fl.A + 2 * n;
        fl.C = fl.B + 2 * n;
        fl.MU = fl.C + 2 * n;
        fl.D = fl.MU + n;
        fl.G = fl.D + n;
        const auto* in = static_cast<const typename C::raw_t*>(src);
        auto* out = static_cast<typename C::raw_t*>(dst);
        // 16-bit storage with nx even: the gathering passes on x pairs
        constexpr bool kPairs = sizeof(typename C::raw_t) == 2;
        const bool pairs = kPairs && d.nx % 2 == 0;
        const int half = d.nx / 2;
        const int th2 = half >= 128 ? 128 : ((half + 31) / 32) * 32;
        const int chunks2 = (half + th2 - 1) / th2;
        constexpr int kRpb = 2;  // rows per block of the forced step (the next one prefetched)
        const unsigned blocks2 = (unsigned)(((d.rows + kRpb - 1) / kRpb) * chunks2);
        if constexpr (kPairs) {
            if (pairs) k_ni_density2x<C><<<(unsigned)(d.rows * chunks2), th2, 0, st>>>(in, d, chunks2, *K, e, fl);
        }
        if (!pairs) k_ni_density<C><<<blocks, kNiThreads, 0, st>>>(in, d, chunks, *K, e, fl);
        // FP32 fields with nx even: the stencil passes on x pairs, in 128-thread blocks
        bool pair_fields = false;
        if constexpr (sizeof(R) == 4) {
            if (d.nx % 2 == 0) {
                const int chunks_f = (half + kNiThreads - 1) / kNiThreads;
                const unsigned blocks_f = (unsigned)(d.rows * chunks_f);
                k_ni_fields2x<R><<<blocks_f, kNiThreads, 0, st>>>(d, chunks_f, fl);
                k_ni_force2x<R><<<blocks_f, kNiThreads, 0, st>>>(d, chunks_f, e, fl);
                pair_fields = true;
            }
        }
        if (!pair_fields) {
            k_ni_fields<R><<<blocks, kNiThreads, 0, st>>>(d, chunks, fl);
            k_ni_force<R><<<blocks, kNiThreads, 0, st>>>(d, chunks, e, fl);
        }
        if constexpr (kPairs) {
            if (pairs)
                k_ni_step2x<C><<<blocks2, th2, 0, st>>>(in, out, d, chunks2, kRpb, *K, (float)twobeta,
                                                         (float)(1.0 / c.theta0), fl.G, err);
        }
        if (!pairs)
            k_ni_step<C><<<blocks, kNiThreads, 0, st>>>(in, out, d, chunks, *K, (R)twobeta, (R)(1.0 / c.theta0), fl.G,
                                                         err);
        return cudaGetLastError();
    });
}

}  // namespace gblb
