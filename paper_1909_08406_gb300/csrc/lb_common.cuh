// Shared device code of the RD3Q41 solver: the velocity table, the storage
// codecs and the fused per-node collision (moments, energy-conserving
// equilibrium, BGK relaxation).
//
// Model: arXiv:1909.08406.  Velocity shells and weights: Sec. IV, Table I.
// Moments: Sec. II.  Rest-state equilibrium to O(eta^3) and the velocity
// series Eq. (feqGenU3): Sec. V.  BGK update: Sec. II.
//
// The per-node arithmetic is organised around the +-c pairs of the velocity
// set: for a pair the equilibrium splits into an even part (shared) and an odd
// part (sign-flipped), so each pair costs one dot product, a handful of FMAs
// and two relaxations.  All shell-dependent quantities are folded into six
// per-node shell constants.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>
#include <utility>

namespace gblb {

constexpr int kQ = 41;
constexpr int kShells = 6;  // rest, sc-1, sc-2, fcc-1, bcc-1, bcc-1/2

// Doubled velocity components 2 c_i, ordered rest then +-c pairs (2k+1, 2k+2).
struct Vel {
    int x, y, z, shell;
};

__host__ __device__ constexpr Vel vel(int i) {
    constexpr Vel t[kQ] = {
        {0, 0, 0, 0},
        // sc-1
        {2, 0, 0, 1}, {-2, 0, 0, 1}, {0, 2, 0, 1}, {0, -2, 0, 1}, {0, 0, 2, 1}, {0, 0, -2, 1},
        // sc-2
        {4, 0, 0, 2}, {-4, 0, 0, 2}, {0, 4, 0, 2}, {0, -4, 0, 2}, {0, 0, 4, 2}, {0, 0, -4, 2},
        // fcc-1
        {2, 2, 0, 3}, {-2, -2, 0, 3}, {2, -2, 0, 3}, {-2, 2, 0, 3},
        {2, 0, 2, 3}, {-2, 0, -2, 3}, {2, 0, -2, 3}, {-2, 0, 2, 3},
        {0, 2, 2, 3}, {0, -2, -2, 3}, {0, 2, -2, 3}, {0, -2, 2, 3},
        // bcc-1
        {2, 2, 2, 4}, {-2, -2, -2, 4}, {2, 2, -2, 4}, {-2, -2, 2, 4},
        {2, -2, 2, 4}, {-2, 2, -2, 4}, {-2, 2, 2, 4}, {2, -2, -2, 4},
        // bcc-1/2
        {1, 1, 1, 5}, {-1, -1, -1, 5}, {1, 1, -1, 5}, {-1, -1, 1, 5},
        {1, -1, 1, 5}, {-1, 1, -1, 5}, {-1, 1, 1, 5}, {1, -1, -1, 5},
    };
    return t[i];
}

// The velocity table as data, for lookups with a run-time index.
struct VelTable {
    Vel v[kQ];
};
__host__ __device__ constexpr VelTable make_vel_table() {
    VelTable t{};
    for (int i = 0; i < kQ; ++i) t.v[i] = vel(i);
    return t;
}
static __constant__ VelTable c_vel = make_vel_table();

// Per-shell lattice constants in the compute type.
template <class R>
struct Consts {
    R w[kShells];    // weight of one velocity of the shell
    R c2[kShells];   // c^2 of the shell
    R p1[kShells];   // rest equilibrium f~/(w rho) = 1 + eta p1 + eta^2 p2 + eta^3 p3
    R p2[kShells];
    R p3[kShells];
    // Shell sums of the momentum projection as cubics in eta: with R_s = f~_s / (w_s rho) and
    // n2, n4, n22 the sums over shell s of c_x^2, c_x^4, c_x^2 c_y^2,
    //   pj[0](eta) = sum_s w_s n2_s R_s,       pj[1](eta) = sum_s w_s n2_s c_s^2 R_s,
    //   pj[2](eta) = sum_s w_s n4_s R_s,       pj[3](eta) = sum_s w_s n22_s R_s,
    // pj[j](eta) = pj[j][0] + eta (pj[j][1] + eta (pj[j][2] + eta pj[j][3])).
    R pj[4][4];
    R n2[kShells];   // sum over the shell of c_x^2 (the packed two-node path sums the shells directly)
    R n4[kShells];   // sum over the shell of c_x^4
    R n22[kShells];  // sum over the shell of c_x^2 c_y^2
    R m2[4];         // M_2  (1+eta)^2 = m2[0] + m2[1] eta + m2[2] eta^2 + m2[3] eta^3
    R m2p[4];        // M_2' (1+eta)^2 likewise
    R theta0;
    R inv_3theta0;
};

template <int... Is, class F>
__device__ __forceinline__ void static_for_impl(std::integer_sequence<int, Is...>, F&& f) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(std::make_integer_sequence<int, N>{}, f);
}

// ---------------------------------------------------------------------------
// Storage codecs.  value(): stored element -> working value v (f, or
// kScale * h); dev(v, w / kScale): deviation f - w; relax(): new working value
// from v and x = 2 beta kScale h^eq; to_raw(): rounding to the storage type.
// ---------------------------------------------------------------------------
struct CodecF64 {  // stores f_i
    using raw_t = double;
    using R = double;
    using KS = double;  // type of the lattice constants
    static constexpr bool stores_f = true;
    static constexpr double kScale = 1.0;
    static __device__ __forceinline__ R value(raw_t r) { return r; }
    static __device__ __forceinline__ R dev(R v, R w) { return v - w; }
    static __device__ __forceinline__ R relax(R v, R omb, R x, R w, R tb) { return fma(omb, v, w * (tb + x)); }
    static __device__ __forceinline__ raw_t to_raw(R v) { return v; }
};

struct CodecF32 {  // stores h_i = f_i / w_i - 1
    using raw_t = float;
    using R = float;
    using KS = float;
    static constexpr bool stores_f = false;
    static constexpr double kScale = 1.0;
    using pair_t = float2;
    static __device__ __forceinline__ pair_t pack2(raw_t a, raw_t b) { return make_float2(a, b); }
    static __device__ __forceinline__ float2 unpack2(pair_t p) { return p; }
    static __device__ __forceinline__ R value(raw_t r) { return r; }
    static __device__ __forceinline__ R dev(R v, R w) { return w * v; }
    static __device__ __forceinline__ R relax(R v, R omb, R x, R, R) { return fmaf(omb, v, x); }
    static __device__ __forceinline__ raw_t to_raw(R v) { return v; }
};

// FP16 stores 2^8 h_i: the power-of-two scale is exact and moves FP16's
// subnormal range (|x| < 6.1e-5) down to |h| < 2.4e-7, while |h| up to 255
// stays finite.  The scale is folded into the per-shell constants, so the
// working value v is the stored (scaled) number.
struct CodecF16 {
    using raw_t = __half;
    using R = float;
    using KS = float;
    static constexpr bool stores_f = false;
    static constexpr double kScale = 256.0;
    static __device__ __forceinline__ R value(raw_t r) { return __half2float(r); }
    static __device__ __forceinline__ R dev(R v, R w) { return w * v; }
    static __device__ __forceinline__ R relax(R v, R omb, R x, R, R) { return fmaf(omb, v, x); }
    static __device__ __forceinline__ raw_t to_raw(R v) { return __float2half_rn(v); }
    // two stored elements kept packed in one register
    using pair_t = __half2;
    static __device__ __forceinline__ pair_t pack2(raw_t a, raw_t b) { return __halves2half2(a, b); }
    static __device__ __forceinline__ float2 unpack2(pair_t p) { return __half22float2(p); }
    // (hi of a, lo of b): the pair that starts at an odd element between two aligned pairs
    static __device__ __forceinline__ pair_t straddle(pair_t a, pair_t b) {
        return __halves2half2(__high2half(a), __low2half(b));
    }
    static __device__ __forceinline__ pair_t to_raw2(float2 v) { return __float22half2_rn(v); }
};

struct CodecBF16 {
    using raw_t = __nv_bfloat16;
    using R = float;
    using KS = float;
    static constexpr bool stores_f = false;
    static constexpr double kScale = 1.0;
    static __device__ __forceinline__ R value(raw_t r) { return __bfloat162float(r); }
    static __device__ __forceinline__ R dev(R v, R w) { return w * v; }
    static __device__ __forceinline__ R relax(R v, R omb, R x, R, R) { return fmaf(omb, v, x); }
    static __device__ __forceinline__ raw_t to_raw(R v) { return __float2bfloat16_rn(v); }
    using pair_t = __nv_bfloat162;
    static __device__ __forceinline__ pair_t pack2(raw_t a, raw_t b) { return __halves2bfloat162(a, b); }
    static __device__ __forceinline__ float2 unpack2(pair_t p) { return __bfloat1622float2(p); }
    static __device__ __forceinline__ pair_t straddle(pair_t a, pair_t b) {
        return __halves2bfloat162(__high2bfloat16(a), __low2bfloat16(b));
    }
    static __device__ __forceinline__ pair_t to_raw2(float2 v) { return __float22bfloat162_rn(v); }
};

// ---------------------------------------------------------------------------
// Two nodes per thread: F2 carries one float per node and maps every
// arithmetic operation onto Blackwell's packed FP32x2 instructions
// (__fadd2_rn, __fmul2_rn, __ffma2_rn; each lane rounds exactly as the scalar
// FP32 operation does), halving the FP32 instruction count of the collision.
// ---------------------------------------------------------------------------
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(double s) : v(make_float2((float)s, (float)s)) {}
    __device__ __forceinline__ F2(int s) : v(make_float2((float)s, (float)s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ F2(float2 x) : v(x) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) {
    a = a + b;
    return a;
}
using ::fma;  // keep the scalar overloads visible next to the F2 one
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

// Reciprocals of the node scalars (1/rho, theta0/theta, ...).  FP64 keeps the IEEE
// division; the FP32 paths use the hardware reciprocal approximation (within 2 ulp),
// far below the FP32 rounding of the populations themselves.
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ F2 recip(F2 x) { return F2(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y)); }

// Two-node codec over a one-node storage codec: same storage, F2 arithmetic.
template <class Base>
struct Codec2 {
    using raw_t = typename Base::raw_t;
    using R = F2;
    using KS = float;
    static constexpr bool stores_f = Base::stores_f;
    static constexpr double kScale = Base::kScale;
    static __device__ __forceinline__ F2 dev(F2 v, F2 w) { return w * v; }
    static __device__ __forceinline__ F2 relax(F2 v, F2 omb, F2 x, F2, F2) { return fma(omb, v, x); }
};

// Moments of one node from the deviations d_i = f_i - w_i (Sec. II):
// drho = rho - 1, j = rho u, dk = <f, c^2> - 3 theta_0.
template <class R>
struct NodeMoments {
    R drho, jx, jy, jz, dk;
};

// dget(I) returns d_I for a compile-time population index I.
template <class R, class G>
__device__ __forceinline__ NodeMoments<R> moments_from(G&& dget) {
    NodeMoments<R> m;
    m.drho = dget(std::integral_constant<int, 0>{});
    m.jx = R(0);
    m.jy = R(0);
    m.jz = R(0);
    m.dk = R(0);
    static_for<20>([&](auto K) {
        constexpr int ip = 2 * K + 1, im = 2 * K + 2;
        constexpr Vel c = vel(ip);
        const R dp = dget(std::integral_constant<int, ip>{});
        const R dm = dget(std::integral_constant<int, im>{});
        const R s = dp + dm;
        const R df = dp - dm;
        m.drho += s;
        // c2 components are doubled: c = c2 / 2
        if constexpr (c.x != 0) m.jx = fma(R(0.5 * c.x), df, m.jx);
        if constexpr (c.y != 0) m.jy = fma(R(0.5 * c.y), df, m.jy);
        if constexpr (c.z != 0) m.jz = fma(R(0.5 * c.z), df, m.jz);
        constexpr double csq = 0.25 * (c.x * c.x + c.y * c.y + c.z * c.z);
        m.dk = fma(R(csq), s, m.dk);
    });
    return m;
}

template <class R>
__device__ __forceinline__ NodeMoments<R> moments_from_dev(const R (&d)[kQ]) {
    return moments_from<R>([&](auto I) { return d[I]; });
}

// Primitive variables of a node: rho, u, eta = theta / theta_0 - 1.
template <class R>
struct NodeState {
    R drho, rho, ux, uy, uz, eta;
};

template <class R, class KS>
__device__ __forceinline__ NodeState<R> state_from_moments(const NodeMoments<R>& m, const Consts<KS>& K) {
    NodeState<R> st;
    st.drho = m.drho;
    st.rho = R(1) + m.drho;
    const R inv_rho = recip(st.rho);
    st.ux = m.jx * inv_rho;
    st.uy = m.jy * inv_rho;
    st.uz = m.jz * inv_rho;
    const R usq = st.ux * st.ux + st.uy * st.uy + st.uz * st.uz;
    // theta = (<f,c^2>/rho - u^2)/3  =>  eta = (dk - 3 theta0 drho - rho u^2) / (3 theta0 rho)
    st.eta = (m.dk - R(3) * K.theta0 * m.drho - st.rho * usq) * inv_rho * K.inv_3theta0;
    return st;
}

template <class R>
__device__ __forceinline__ bool state_ok(const NodeState<R>& st) {
    // rho > 0, theta > 0 and both finite (NaN fails every comparison)
    return st.rho > R(0) && st.rho < R(1e30) && st.eta > R(-1) && st.eta < R(1e30) && st.ux == st.ux &&
           st.uy == st.uy && st.uz == st.uz && fabs(st.ux) < R(1e30) && fabs(st.uy) < R(1e30) &&
           fabs(st.uz) < R(1e30);
}

// Two nodes: rho > 0, theta > 0 and |rho| + |eta| + |u_x| + |u_y| + |u_z| below 1e30 for both (a NaN
// or an infinity in any of them fails the last comparison).
__device__ __forceinline__ bool state_ok(const NodeState<F2>& st) {
    const float ma = st.rho.v.x + st.eta.v.x + fabsf(st.ux.v.x) + fabsf(st.uy.v.x) + fabsf(st.uz.v.x);
    const float mb = st.rho.v.y + st.eta.v.y + fabsf(st.ux.v.y) + fabsf(st.uy.v.y) + fabsf(st.uz.v.y);
    return st.rho.v.x > 0.f && st.rho.v.y > 0.f && st.eta.v.x > -1.f && st.eta.v.y > -1.f && ma < 1e30f &&
           mb < 1e30f;
}

// Equilibrium (Eq. feqGenU3, with the optional momentum projection) and BGK
// relaxation of one node.  v[i] are the working values of the node's incoming
// populations (f or h, see the codec), tb = 2 beta, omb = 1 - 2 beta.
// sink(I, value) receives the new working value of population I.
template <class Codec, bool PROJECT, class VGet, class Sink>
__device__ __forceinline__ void equilibrium_relax_g(const NodeState<typename Codec::R>& st,
                                                    const Consts<typename Codec::KS>& K, typename Codec::R tb,
                                                    typename Codec::R omb, VGet&& vget, Sink&& sink) {
    using R = typename Codec::R;
    const R rho = st.rho, eta = st.eta;
    const R inv_1pe = recip(R(1) + eta);             // theta_0 / theta
    const R inv_theta = inv_1pe / K.theta0;          // 1 / theta
    const R usq = st.ux * st.ux + st.uy * st.uy + st.uz * st.uz;
    const R g = usq * inv_theta;                     // u^2 / theta
    // M_2, M_2' from their exact polynomials; A_1, A_2 (Sec. V)
    const R r2 = inv_1pe * inv_1pe;
    const R M2 = (K.m2[0] + eta * (K.m2[1] + eta * (K.m2[2] + eta * K.m2[3]))) * r2;
    const R M2p = (K.m2p[0] + eta * (K.m2p[1] + eta * (K.m2p[2] + eta * K.m2p[3]))) * r2;
    const R A1 = R(2.5) * M2 * recip(R(1) + R(2.5) * M2);
    const R A2 = R(5) * A1 * (R(1) - M2) - (R(3) + M2p - R(5) * M2);
    // rest-state factors per shell: f~_s = w_s rho R_s, R_s - 1 = eta (p1 + eta (p2 + eta p3));
    // per-shell even constant C_s and odd factor D_s of the series
    //   X_i = C_s + a^2/2 + a D_s + a^3/6,  a = u.c/theta
    //   C_s = -g (1 - A1)/2 - g c_s^2 A1 / (6 theta),  D_s = 1 + g A2 / 6 - g c_s^2 A1 / (6 theta)
    // They are formed where a shell is used (the populations are ordered by shell), which keeps
    // only one shell's factors live at a time.
    const R gA1_6t = g * A1 * inv_theta * R(1.0 / 6.0);
    const R cg = R(-0.5) * g * (R(1) - A1);
    const R dg = g * A2 * R(1.0 / 6.0);
    auto rest_m1 = [&](int s) { return eta * (K.p1[s] + eta * (K.p2[s] + eta * K.p3[s])); };
    auto dm1 = [&](int s) { return dg - gA1_6t * K.c2[s]; };
    const R upx = st.ux * inv_theta, upy = st.uy * inv_theta, upz = st.uz * inv_theta;
    // momentum projection v = dj / (rho theta), dj = rho u - sum_i f^eq_i c_i in closed form:
    //   dj_a = -(u_a/theta) S - [S4 u_a^3 + 3 S22 u_a (u^2 - u_a^2)] / (6 theta^3), with the shell sums
    //   S = sum_s f~_s n2_s (D_s - 1) = rho [dg pj[0] - (g A1 / 6 theta) pj[1]], S4 = rho pj[2],
    //   S22 = rho pj[3] (f~_s = w_s rho R_s, D_s - 1 = dg - (g A1 / 6 theta) c_s^2)
    R vx = R(0), vy = R(0), vz = R(0);
    if constexpr (PROJECT) {
        R S, S4, S22;
        if constexpr (std::is_same<R, F2>::value) {
            // packed two-node arithmetic: the shell sums term by term (measured faster here than the
            // cubics, which lengthen the packed path's dependency chains)
            S = R(0);
            S4 = R(0);
            S22 = R(0);
#pragma unroll
            for (int s = 1; s < kShells; ++s) {
                const R ft = K.w[s] * (rho + rho * rest_m1(s));
                S = fma(ft * K.n2[s], dm1(s), S);
                S4 = fma(ft, K.n4[s], S4);
                S22 = fma(ft, K.n22[s], S22);
            }
        } else {
            auto pj = [&](int j) { return K.pj[j][0] + eta * (K.pj[j][1] + eta * (K.pj[j][2] + eta * K.pj[j][3])); };
            S = rho * (dg * pj(0) - gA1_6t * pj(1));
            S4 = rho * pj(2);
            S22 = rho * pj(3);
        }
        const R it3 = inv_theta * inv_theta * inv_theta * R(1.0 / 6.0);
        const R ux2 = st.ux * st.ux, uy2 = st.uy * st.uy, uz2 = st.uz * st.uz;
        const R djx = -upx * S - it3 * st.ux * (S4 * ux2 + R(3) * S22 * (usq - ux2));
        const R djy = -upy * S - it3 * st.uy * (S4 * uy2 + R(3) * S22 * (usq - uy2));
        const R djz = -upz * S - it3 * st.uz * (S4 * uz2 + R(3) * S22 * (usq - uz2));
        const R k = inv_theta * recip(rho);
        vx = djx * k;
        vy = djy * k;
        vz = djz * k;
    }
    // rest population: a = 0
    {
        const R rm1 = rest_m1(0);
        const R P0 = tb * (rho + rho * rm1);
        const R x0 = fma(P0, cg - gA1_6t * K.c2[0], tb * (st.drho + rho * rm1));
        sink(std::integral_constant<int, 0>{},
             Codec::relax(vget(std::integral_constant<int, 0>{}), omb, x0, K.w[0], tb));
    }
    R P, B, Ds;  // factors of the current shell
    static_for<20>([&](auto KK) {
        constexpr int ip = 2 * KK + 1, im = 2 * KK + 2;
        constexpr Vel c = vel(ip);
        constexpr int s = c.shell;
        if constexpr (KK == 0 || vel(ip - 2).shell != s) {
            const R rm1 = rest_m1(s);
            P = tb * (rho + rho * rm1);
            B = fma(P, cg - gA1_6t * K.c2[s], tb * (st.drho + rho * rm1));
            Ds = R(1) + dm1(s);
        }
        // p_s = D_s u / theta + v
        R a = R(0), q = R(0);
        if constexpr (c.x != 0) {
            a = fma(R(0.5 * c.x), upx, a);
            q = fma(R(0.5 * c.x), fma(Ds, upx, vx), q);
        }
        if constexpr (c.y != 0) {
            a = fma(R(0.5 * c.y), upy, a);
            q = fma(R(0.5 * c.y), fma(Ds, upy, vy), q);
        }
        if constexpr (c.z != 0) {
            a = fma(R(0.5 * c.z), upz, a);
            q = fma(R(0.5 * c.z), fma(Ds, upz, vz), q);
        }
        const R a2 = a * a;
        const R t = fma(R(0.5) * P, a2, B);
        const R o = fma(P * R(1.0 / 6.0), a2 * a, P * q);
        sink(std::integral_constant<int, ip>{},
             Codec::relax(vget(std::integral_constant<int, ip>{}), omb, t + o, K.w[s], tb));
        sink(std::integral_constant<int, im>{},
             Codec::relax(vget(std::integral_constant<int, im>{}), omb, t - o, K.w[s], tb));
    });
}

__device__ __forceinline__ double expm1_of(double x) { return expm1(x); }
__device__ __forceinline__ float expm1_of(float x) { return expm1f(x); }

__device__ __forceinline__ double log1p_of(double x) { return log1p(x); }
__device__ __forceinline__ float log1p_of(float x) { return log1pf(x); }

// phi(y) = (1 + y) ln(1 + y) - y, the entropy change along the path per unit population.  For
// |y| < 1/8 its series sum_{n >= 2} (-y)^n / (n (n - 1)) (to y^8 in FP32, y^18 in FP64: below
// the unit roundoff of y^2 / 2), else the formula (cancellation at most 16 ulp there).
template <class R>
__device__ __forceinline__ R path_phi(R y) {
    constexpr int N = sizeof(R) == 8 ? 18 : 8;
    if (fabs(y) < R(0.125)) {
        R s = R(0);
#pragma unroll
        for (int n = N; n >= 2; --n) s = fma(s, -y, R(1.0 / (n * (n - 1.0))));
        return s * y * y;
    }
    return (R(1) + y) * log1p_of(y) - y;
}

// Entropic path length alpha of one node (Sec. "Droplet Collision": the update with alpha beta,
// alpha such that the H theorem holds, from x_i = f^eq_i / f_i - 1): the nontrivial root of
// Delta H(alpha) = H(f + alpha (f^eq - f)) - H(f), H = sum_i f_i ln(f_i / w_i).  For an f^eq
// with the moments of f whose logarithm is a sum of collision invariants (the exact entropic
// equilibrium: ln(f^eq_i / w_i) = ln rho + X_i), sum_i f_i x_i (1 + ln(f^eq_i / w_i)) vanishes
// and, with ln(f_i / w_i) = ln(f^eq_i / w_i) - ln(1 + x_i),
//   Delta H(alpha) = sum_i f_i [phi(alpha x_i) - alpha x_i ln(1 + x_i)],
//   d/dalpha     = sum_i f_i x_i [ln(1 + alpha x_i) - ln(1 + x_i)],
// both free of cancellation as x -> 0 (alpha -> 2).  Newton from 2, kept inside (0, alpha_max),
// alpha_max = min over x_i < 0 of -1/x_i; left of Delta H's minimum it doubles alpha instead.
// fw[i] = f_i / w_i, lx[i] = ln(1 + x_i).  Returns 2 (plain BGK) when f = f^eq or when Newton
// does not converge (no root below alpha_max).
template <class R>
__device__ __forceinline__ R entropic_path(const Consts<R>& K, const R (&x)[kQ], const R (&lx)[kQ],
                                           const R (&fw)[kQ]) {
    constexpr bool kDouble = sizeof(R) == 8;
    constexpr int MAXIT = kDouble ? 40 : 30;
    const R tol = kDouble ? R(1e-14) : R(1e-6);
    R amax = R(0), xmax = R(0);  // amax as 1 / alpha_max = max over i of -x_i
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        amax = fmax(amax, -x[i]);
        xmax = fmax(xmax, fabs(x[i]));
    }
    if (!(xmax > R(0))) return R(2);
    const bool bounded = amax > R(0);
    const R alim = bounded ? R(1) / amax : R(0);
    R a = (!bounded || alim > R(2)) ? R(2) : R(0.5) * alim;
    bool conv = false;
#pragma unroll 1
    for (int it = 0; it < MAXIT; ++it) {
        R g = R(0), dg = R(0);
        static_for<kQ>([&](auto I) {
            const R f = K.w[vel(I).shell] * fw[I], y = a * x[I];
            g = fma(f, path_phi(y) - y * lx[I], g);
            dg = fma(f * x[I], log1p_of(y) - lx[I], dg);
        });
        R an;
        if (!(dg > R(0)))
            an = (!bounded || R(2) * a < alim) ? R(2) * a : R(0.5) * (a + alim);
        else
            an = a - g / dg;
        if (bounded && !(an < alim)) an = R(0.5) * (a + alim);
        if (!(an > R(0))) an = R(0.5) * a;
        conv = dg > R(0) && fabs(an - a) <= tol * an;
        a = an;
        if (conv) break;
    }
    return conv ? a : R(2);
}

// Exact entropic equilibrium (Eqs. (discreteentropiceq) and
// (fivelagrangemultipliersystem)) and BGK relaxation of one node.
//   f^eq_i = w_i rho exp(X_i),  X_i = l0 + l.c_i + l4 (c_i^2 - 3 theta_0),
// with the five multipliers fixed by <f^eq, (1, c, c^2)> = (rho, rho u,
// rho u^2 + 3 rho theta).  Divided by rho and written for the deviations this
// is  sum_i w_i expm1(X_i) phi_i = t,  phi = (1, c, c^2 - 3 theta_0),
// t = (0, u, u^2 + 3 theta_0 eta), which keeps full relative precision of the
// small deviations in FP32.  Newton's method starts from the solution of the
// linearised system (J = diag(1, theta_0, theta_0, theta_0, 6 theta_0^2) at
// rest); once the residual is below `tol` one more step is taken (quadratic
// convergence then leaves round-off), and `ok` is cleared if that does not
// happen within MAXIT steps.  The working value passed on is x_i = tb h^eq_i
// with h^eq_i = rho expm1(X_i) + (rho - 1).
// PATH: the relaxation factor 2 beta becomes alpha beta with the entropic path length alpha of
// entropic_path (tb and 1 - omb scaled by alpha / 2).
template <class Codec, bool PATH = false, class VGet, class Sink>
__device__ __forceinline__ void entropic_relax(const NodeState<typename Codec::R>& st,
                                               const Consts<typename Codec::KS>& K, typename Codec::R tb,
                                               typename Codec::R omb, VGet&& vget, Sink&& sink, bool& ok) {
    using R = typename Codec::R;
    constexpr bool kDouble = sizeof(R) == 8;
    constexpr int MAXIT = kDouble ? 20 : 12;
    const R tol = kDouble ? R(1e-10) : R(3e-5);
    const R th0 = K.theta0;
    const R usq = st.ux * st.ux + st.uy * st.uy + st.uz * st.uz;
    const R t4 = usq + R(3) * th0 * st.eta;
    R l[5] = {R(0), st.ux / th0, st.uy / th0, st.uz / th0, t4 / (R(6) * th0 * th0)};
    const R tgt[5] = {R(0), st.ux, st.uy, st.uz, t4};
    bool conv = false;
#pragma unroll 1
    for (int it = 0; it < MAXIT; ++it) {
        // residual F and Jacobian J (upper triangle, row-major) at l
        R F[5] = {R(0), R(0), R(0), R(0), R(0)};
        R J[15] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
        {
            const R p4 = K.c2[0] - R(3) * th0;
            const R em = expm1_of(l[0] + l[4] * p4);
            const R w = K.w[0], ex = em + R(1);
            F[0] += w * em;
            F[4] += w * p4 * em;
            J[0] += w * ex;
            J[4] += w * p4 * ex;
            J[14] += w * p4 * p4 * ex;
        }
        static_for<20>([&](auto KK) {
            constexpr Vel c = vel(2 * KK + 1);
            constexpr double cx = 0.5 * c.x, cy = 0.5 * c.y, cz = 0.5 * c.z;
            const R w = K.w[c.shell], p4 = K.c2[c.shell] - R(3) * th0;
            const R E = l[0] + l[4] * p4;
            R O = R(0);
            if constexpr (cx != 0) O += R(cx) * l[1];
            if constexpr (cy != 0) O += R(cy) * l[2];
            if constexpr (cz != 0) O += R(cz) * l[3];
            const R ep = expm1_of(E + O), emn = expm1_of(E - O);
            const R se = w * (ep + emn), de = w * (ep - emn);  // even / odd parts
            const R sx = se + R(2) * w;                        // w (exp(E+O) + exp(E-O))
            const R cc[3] = {R(cx), R(cy), R(cz)};
            F[0] += se;
            F[4] += p4 * se;
            J[0] += sx;
            J[4] += p4 * sx;
            J[14] += p4 * p4 * sx;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                F[1 + a] += cc[a] * de;
                J[1 + a] += cc[a] * de;          // (0, 1+a)
                J[(a == 0 ? 8 : a == 1 ? 11 : 13)] += cc[a] * p4 * de;  // (1+a, 4)
            }
            // (1+a, 1+b), b >= a: 5 6 7 / 9 10 / 12
            J[5] += cc[0] * cc[0] * sx;
            J[6] += cc[0] * cc[1] * sx;
            J[7] += cc[0] * cc[2] * sx;
            J[9] += cc[1] * cc[1] * sx;
            J[10] += cc[1] * cc[2] * sx;
            J[12] += cc[2] * cc[2] * sx;
        });
        R res = R(0);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            F[k] -= tgt[k];
            res = fmax(res, fabs(F[k]));
        }
        conv = res <= tol;  // false for NaN
        // solve J d = -F (symmetric positive definite: elimination without pivoting)
        R A[5][5];
        {
            int q = 0;
#pragma unroll
            for (int r = 0; r < 5; ++r)
#pragma unroll
                for (int cix = r; cix < 5; ++cix) {
                    A[r][cix] = J[q];
                    A[cix][r] = J[q];
                    ++q;
                }
        }
        R b[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) b[k] = -F[k];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const R inv = R(1) / A[k][k];
#pragma unroll
            for (int r = k + 1; r < 5; ++r) {
                const R f = A[r][k] * inv;
#pragma unroll
                for (int cix = k; cix < 5; ++cix) A[r][cix] -= f * A[k][cix];
                b[r] -= f * b[k];
            }
        }
#pragma unroll
        for (int k = 4; k >= 0; --k) {
            R sum = b[k];
#pragma unroll
            for (int cix = k + 1; cix < 5; ++cix) sum -= A[k][cix] * b[cix];
            b[k] = sum / A[k][k];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) l[k] += b[k];
        if (conv) break;
    }
    if (!conv) ok = false;
    if constexpr (PATH) {
        // h_i and x_i = f^eq_i / f_i - 1 = (h^eq_i - h_i) / (1 + h_i), h^eq = rho expm1(X) + drho
        auto h_of = [&](auto I) {
            if constexpr (Codec::stores_f)
                return vget(I) / K.w[vel(I).shell] - R(1);
            else
                return vget(I) * R(1.0 / Codec::kScale);
        };
        R x[kQ], lx[kQ], fw[kQ];
        auto set_x = [&](auto I, R heq) {
            const R h = h_of(I);
            fw[I] = R(1) + h;
            x[I] = (heq - h) / fw[I];
            lx[I] = log1p_of(x[I]);
        };
        set_x(std::integral_constant<int, 0>{}, st.rho * expm1_of(l[0] + l[4] * (K.c2[0] - R(3) * th0)) + st.drho);
        static_for<20>([&](auto KK) {
            constexpr int ip = 2 * KK + 1, im = 2 * KK + 2;
            constexpr Vel c = vel(ip);
            const R E = l[0] + l[4] * (K.c2[c.shell] - R(3) * th0);
            R O = R(0);
            if constexpr (c.x != 0) O += R(0.5 * c.x) * l[1];
            if constexpr (c.y != 0) O += R(0.5 * c.y) * l[2];
            if constexpr (c.z != 0) O += R(0.5 * c.z) * l[3];
            set_x(std::integral_constant<int, ip>{}, st.rho * expm1_of(E + O) + st.drho);
            set_x(std::integral_constant<int, im>{}, st.rho * expm1_of(E - O) + st.drho);
        });
        const R half_alpha = R(0.5) * entropic_path<R>(K, x, lx, fw);
        const R tba = tb * half_alpha, omba = R(1) - (R(1) - omb) * half_alpha;
        // relaxation towards h^eq = h + x (1 + h)
        static_for<kQ>([&](auto I) {
            const R heq = fma(x[I], fw[I], h_of(I));
            sink(I, Codec::relax(vget(I), omba, tba * heq, K.w[vel(I).shell], tba));
        });
        return;
    }
    // relaxation towards h^eq = rho expm1(X) + drho
    {
        const R em = expm1_of(l[0] + l[4] * (K.c2[0] - R(3) * th0));
        sink(std::integral_constant<int, 0>{},
             Codec::relax(vget(std::integral_constant<int, 0>{}), omb, tb * (st.rho * em + st.drho), K.w[0], tb));
    }
    static_for<20>([&](auto KK) {
        constexpr int ip = 2 * KK + 1, im = 2 * KK + 2;
        constexpr Vel c = vel(ip);
        const R E = l[0] + l[4] * (K.c2[c.shell] - R(3) * th0);
        R O = R(0);
        if constexpr (c.x != 0) O += R(0.5 * c.x) * l[1];
        if constexpr (c.y != 0) O += R(0.5 * c.y) * l[2];
        if constexpr (c.z != 0) O += R(0.5 * c.z) * l[3];
        sink(std::integral_constant<int, ip>{},
             Codec::relax(vget(std::integral_constant<int, ip>{}), omb, tb * (st.rho * expm1_of(E + O) + st.drho),
                          K.w[c.shell], tb));
        sink(std::integral_constant<int, im>{},
             Codec::relax(vget(std::integral_constant<int, im>{}), omb, tb * (st.rho * expm1_of(E - O) + st.drho),
                          K.w[c.shell], tb));
    });
}

// Equilibrium kinds: 0 = Eq. (feqGenU3) as printed, 1 = with the momentum
// projection, 2 = the exact entropic equilibrium (clears `ok` if Newton fails),
// 3 = that equilibrium with the entropic path length (entropic_path).
template <class Codec, int EQ, class Sink>
__device__ __forceinline__ void equilibrium_relax(const NodeState<typename Codec::R>& st,
                                                  const Consts<typename Codec::KS>& K, typename Codec::R tb,
                                                  typename Codec::R omb, const typename Codec::R (&v)[kQ], Sink&& sink,
                                                  bool& ok) {
    if constexpr (EQ == 2 || EQ == 3)
        entropic_relax<Codec, EQ == 3>(st, K, tb, omb, [&](auto I) { return v[I]; }, sink, ok);
    else
        equilibrium_relax_g<Codec, EQ == 1>(st, K, tb, omb, [&](auto I) { return v[I]; }, sink);
}

// ---------------------------------------------------------------------------
// Stochastic rounding of the BF16 store (lb_set_stochastic_rounding).  A BF16
// number is the upper half of an FP32 bit pattern; adding 16 uniform random
// bits r to the lower half and truncating rounds the magnitude up with
// probability (lower half) / 2^16, so the stored value is unbiased:
//   SR(v; r) = upper half of (bits(v) + r).
// The bits come from a counter-based generator:
//   step key    k_t = H(H(lo(seed) ^ H(hi(seed))) + t),  t = steps since enabling
//   node pair   s_0 = H(k_t ^ (q >> 1)),  q = s nx ny nz + (z ny + y) nx + x
//   population  s_(i+1) = 1664525 s_i + 1013904223 (mod 2^32), i = 0..40 in the
//               library's population order,  w_i = s_(i+1) ^ (s_(i+1) >> 16)
//   r = low 16 bits of w_i for even q, high 16 bits for odd q
// where H is the 32-bit PCG hash of Jarzynski and Olano (Hash Functions for GPU
// Rendering, JCGT 9(3), 2020) and the recurrence is the Numerical Recipes
// linear congruential generator.  The two nodes of an x pair share one word.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr uint32_t pcg_hash(uint32_t x) {
    const uint32_t state = x * 747796405u + 2891336453u;
    const uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
constexpr uint32_t kSrLcgA = 1664525u, kSrLcgC = 1013904223u;
// s_n = sr_lcg_a(n) s_0 + sr_lcg_c(n) after n steps of the recurrence
__host__ __device__ constexpr uint32_t sr_lcg_a(int n) {
    uint32_t a = 1u;
    for (int k = 0; k < n; ++k) a *= kSrLcgA;
    return a;
}
__host__ __device__ constexpr uint32_t sr_lcg_c(int n) {
    uint32_t c = 0u;
    for (int k = 0; k < n; ++k) c = c * kSrLcgA + kSrLcgC;
    return c;
}
inline uint32_t sr_step_key(uint64_t seed, uint32_t t) {
    return pcg_hash(pcg_hash((uint32_t)seed ^ pcg_hash((uint32_t)(seed >> 32))) + t);
}
// w_I of a node pair with first state s0
template <int I>
__device__ __forceinline__ uint32_t sr_word(uint32_t s0) {
    constexpr uint32_t A = sr_lcg_a(I + 1), C = sr_lcg_c(I + 1);
    const uint32_t s = A * s0 + C;
    return s ^ (s >> 16);
}
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float v, uint32_t r16) {
    return __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + r16) >> 16));
}
// the pair (v.x, v.y) of nodes q (even) and q + 1 with one word w
__device__ __forceinline__ __nv_bfloat162 sr_bf16x2(float2 v, uint32_t w) {
    const uint32_t lo = __float_as_uint(v.x) + (w & 0xFFFFu);
    const uint32_t hi = __float_as_uint(v.y) + (w >> 16);
    const uint32_t packed = __byte_perm(lo, hi, 0x7632);
    __nv_bfloat162 r;
    memcpy(&r, &packed, 4);
    return r;
}

// Geometry of one population buffer.
struct Dims {
    int nx, ny, nz;
    int64_t plane;  // nx * ny * nz
    int64_t rows;   // 2 * ny * nz
};

// coordinate of (a) wrapped into [0, n) for a in [-2, n + 1]
__device__ __forceinline__ int wrap(int a, int n) {
    a = a < 0 ? a + n : a;
    a = a < 0 ? a + n : a;
    a = a >= n ? a - n : a;
    a = a >= n ? a - n : a;
    return a;
}

}  // namespace gblb
