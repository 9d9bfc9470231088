// Isothermal nonideal fluid (Sec. "Nonideal Fluids and two-phase flow"; derivative
// stencil of Appendix A), with the van der Waals, the Peng-Robinson type (Eq. cspreos)
// or the Carnahan-Starling equation of state.
//
// Per step, from the post-collision state src:
//   k_ni_density  rho of the streamed populations, sum_i f_i(x - c_i), and
//                 mu_nid(rho), F_nid(rho) of each node
//   k_ni_fields   per node: grad2 rho (3), lap rho, lap F_nid
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
// k_ni_step2x: the x-pair gather of k_step2x, packed FP32x2 arithmetic).
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

// Per-node field records in the compute type F (n = 2 nx ny nz nodes, field index q):
//   P1[q] = {rho, mu, F, 0}                        (density pass)
//   P2[q] = {grad2 rho (3), lap rho}, P3[q] = lap F (field pass)
//   G[a n + q] = g^nid_a                           (force pass)
// A stencil neighbour's values then take three loads.
template <class F>
struct alignas(4 * sizeof(F)) NiRec {
    F x, y, z, w;
};
template <class F>
struct NiFields {
    NiRec<F>* P1;
    NiRec<F>* P2;
    F* P3;
    F* G;
};

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
    m[0] = own + zs + ys + (uint32_t)wrap(x + 1, d.nx);
    m[1] = own + zs + ys + (uint32_t)wrap(x - 1, d.nx);
    m[2] = own + zs + (uint32_t)wrap(y + 1, d.ny) * nx + xs;
    m[3] = own + zs + (uint32_t)wrap(y - 1, d.ny) * nx + xs;
    m[4] = own + (uint32_t)wrap(z + 1, d.nz) * nxy + ys + xs;
    m[5] = own + (uint32_t)wrap(z - 1, d.nz) * nxy + ys + xs;
    const uint32_t X[2] = {(uint32_t)wrap(x + s, d.nx), (uint32_t)wrap(x + s - 1, d.nx)};
    const uint32_t Y[2] = {(uint32_t)wrap(y + s, d.ny) * nx, (uint32_t)wrap(y + s - 1, d.ny) * nx};
    const uint32_t Z[2] = {(uint32_t)wrap(z + s, d.nz) * nxy, (uint32_t)wrap(z + s - 1, d.nz) * nxy};
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
                                                           int chunks, Consts<typename Codec::R> K, NiEos e,
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
    fl.P1[q] = NiRec<R>{r, mu, Fe, R(0)};
}

template <class F>
__global__ void __launch_bounds__(kNiThreads) k_ni_fields(Dims d, int chunks, NiFields<F> fl) {
    int64_t q;
    int s, z, y, x;
    if (!ni_node(d, chunks, q, s, z, y, x)) return;
    const NiRec<F> p0 = fl.P1[q];
    const F r0 = p0.x, F0 = p0.z;
    F g[3] = {F(0), F(0), F(0)}, lr = F(14.0 / 36.0) * r0, lF = F(14.0 / 36.0) * F0;
    uint32_t nb[kStencil];
    ni_neighbors(d, s, z, y, x, nb);
#pragma unroll
    for (int k = 0; k < kStencil; ++k) {
        int cx, cy, cz;
        F w;
        stencil(k, cx, cy, cz, w);
        const NiRec<F> pn = fl.P1[nb[k]];
        const F rn = pn.x;
        g[0] += w * F(0.5 * cx) * rn;
        g[1] += w * F(0.5 * cy) * rn;
        g[2] += w * F(0.5 * cz) * rn;
        lr += w * rn;
        lF += w * pn.z;
    }
    fl.P2[q] = NiRec<F>{g[0] * F(1.0 / kHatTheta), g[1] * F(1.0 / kHatTheta), g[2] * F(1.0 / kHatTheta),
                        F(2.0 / kHatTheta) * (lr - r0)};
    fl.P3[q] = F(2.0 / kHatTheta) * (lF - F0);
}

// g^nid at node q (s, z, y, x) from the fields of its stencil neighbours, into g[3].
template <class F>
__device__ __forceinline__ void ni_force(const Dims& d, const NiEos& e, const NiFields<F>& fl, int64_t q, int s,
                                         int z, int y, int x, F (&g)[3]) {
    F dmu[3] = {0, 0, 0}, dF[3] = {0, 0, 0}, dlF[3] = {0, 0, 0}, divI[3] = {0, 0, 0};
    uint32_t nb[kStencil];
    ni_neighbors(d, s, z, y, x, nb);
#pragma unroll
    for (int k = 0; k < kStencil; ++k) {
        int cx, cy, cz;
        F w;
        stencil(k, cx, cy, cz, w);
        const uint32_t m = nb[k];
        const int cc[3] = {cx, cy, cz};
        const NiRec<F> p1 = fl.P1[m], p2 = fl.P2[m];
        const F lFm = fl.P3[m];
        const F gr[3] = {p2.x, p2.y, p2.z};
        const F iso = F(-0.5) * (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]) - p1.x * p2.w;
        for (int a = 0; a < 3; ++a) {
            if (cc[a] == 0) continue;
            const F wc = w * F(0.5 * cc[a]);
            dmu[a] += wc * p1.y;
            dF[a] += wc * p1.z;
            dlF[a] += wc * lFm;
        }
        // grad2_b I_ab: sum over the stencil of w c_b I_ab(x + c)
        for (int a = 0; a < 3; ++a) {
            F t = 0;
            for (int b = 0; b < 3; ++b) {
                if (cc[b] == 0) continue;
                const F I_ab = gr[a] * gr[b] + (a == b ? iso : F(0));
                t += w * F(0.5 * cc[b]) * I_ab;
            }
            divI[a] += t;
        }
    }
    const NiRec<F> q1 = fl.P1[q], q2 = fl.P2[q];
    const F r0 = q1.x, mu0 = q1.y, inv_th = F(1.0 / kHatTheta);
    const F g2r[3] = {q2.x, q2.y, q2.z};
    for (int a = 0; a < 3; ++a) {
        const F g2mu = dmu[a] * inv_th, g2F = dF[a] * inv_th, g2lF = dlF[a] * inv_th;
        const F g4F = g2F - F(0.5 * kHatTheta) * g2lF;
        const F rg = -(r0 * g2mu + mu0 * g2r[a] - F(e.eta) * g2F - (F(1) - F(e.eta)) * g4F +
                       F(e.kappa) * divI[a] * inv_th);
        g[a] = rg / r0;
    }
}

// g^nid of every node into G (a pass of its own: folded into the step, the stencil sums raise the
// step's register count and the fused step ran slower than the two passes).
template <class F>
__global__ void __launch_bounds__(kNiThreads) k_ni_force(Dims d, int chunks, NiEos e, NiFields<F> fl) {
    int64_t q;
    int s, z, y, x;
    if (!ni_node(d, chunks, q, s, z, y, x)) return;
    F g[3];
    ni_force<F>(d, e, fl, q, s, z, y, x, g);
    const int64_t n = 2 * d.plane;
    for (int a = 0; a < 3; ++a) fl.G[a * n + q] = g[a];
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
// packed FP32x2 arithmetic.  Blocks cover (row, chunk of x pairs), rows (s, z, y); x is the
// thread's even node, q its field index.
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

// k_ni_density for an x pair.
template <class Codec>
__global__ void __launch_bounds__(kStepThreads) k_ni_density2x(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                               int chunks, Consts<float> K, NiEos e,
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
    fl.P1[q] = NiRec<float>{r.v.x, mu0, F0, 0.f};
    fl.P1[q + 1] = NiRec<float>{r.v.y, mu1, F1, 0.f};
}

// k_ni_step for an x pair: the forcing is applied as each population's equilibrium is formed.
template <class Codec>
__global__ void __launch_bounds__(kStepThreads, 3) k_ni_step2x(const typename Codec::raw_t* __restrict__ src,
                                                               typename Codec::raw_t* __restrict__ dst, Dims d,
                                                               int chunks, Consts<float> K, float tb, float inv_theta0,
                                                               const float* __restrict__ G, int* __restrict__ err) {
    using P = typename Codec::pair_t;
    using C2 = Codec2<Codec>;
    uint32_t q;
    int s, z, y, x;
    if (!ni_pair(d, chunks, q, s, z, y, x)) return;
    P pv[kQ];
    ni_gather2x<Codec>(src, d, s, z, y, x, pv);
    auto vget = [&](auto I) { return F2(Codec::unpack2(pv[I])); };
    const size_t n = 2 * (size_t)d.plane;
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

size_t nonideal_doubles(const Dims& d) { return (size_t)12 * 2 * d.plane; }

cudaError_t launch_nonideal_step(int prec, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                                 double twobeta, int kind, const double eos[4], double* work, int* err,
                                 cudaStream_t st) {
    const int64_t n = 2 * d.plane;
    const int chunks = (d.nx + kNiThreads - 1) / kNiThreads;
    const unsigned blocks = (unsigned)(d.rows * chunks);
    if (kind < kVdW || kind > kCarnahanStarling) return cudaErrorInvalidValue;
    const NiEos e{eos[0], eos[1], c.theta0, eos[2], eos[3], kind};
    return ni_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        using R = typename C::R;
        const Consts<R>* K;
        if constexpr (sizeof(R) == 8)
            K = &c.kd;
        else
            K = &c.kf;
        // field records in the compute type: P1, P2 (4 values per node each), P3, G (1 and 3)
        NiFields<R> fl;
        fl.P1 = reinterpret_cast<NiRec<R>*>(work);
        fl.P2 = fl.P1 + n;
        fl.P3 = reinterpret_cast<R*>(fl.P2 + n);
        fl.G = fl.P3 + n;
        const auto* in = static_cast<const typename C::raw_t*>(src);
        auto* out = static_cast<typename C::raw_t*>(dst);
        // 16-bit storage with nx even: the gathering passes on x pairs
        constexpr bool kPairs = sizeof(typename C::raw_t) == 2;
        const bool pairs = kPairs && d.nx % 2 == 0;
        const int half = d.nx / 2;
        const int th2 = half >= 128 ? 128 : ((half + 31) / 32) * 32;
        const int chunks2 = (half + th2 - 1) / th2;
        const unsigned blocks2 = (unsigned)(d.rows * chunks2);
        if constexpr (kPairs) {
            if (pairs) k_ni_density2x<C><<<blocks2, th2, 0, st>>>(in, d, chunks2, *K, e, fl);
        }
        if (!pairs) k_ni_density<C><<<blocks, kNiThreads, 0, st>>>(in, d, chunks, *K, e, fl);
        k_ni_fields<R><<<blocks, kNiThreads, 0, st>>>(d, chunks, fl);
        k_ni_force<R><<<blocks, kNiThreads, 0, st>>>(d, chunks, e, fl);
        if constexpr (kPairs) {
            if (pairs)
                k_ni_step2x<C><<<blocks2, th2, 0, st>>>(in, out, d, chunks2, *K, (float)twobeta,
                                                         (float)(1.0 / c.theta0), fl.G, err);
        }
        if (!pairs)
            k_ni_step<C><<<blocks, kNiThreads, 0, st>>>(in, out, d, chunks, *K, (R)twobeta, (R)(1.0 / c.theta0), fl.G,
                                                         err);
        return cudaGetLastError();
    });
}

}  // namespace gblb
