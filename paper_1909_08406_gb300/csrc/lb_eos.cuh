// Equations of state of the isothermal nonideal fluid (Sec. "Nonideal Fluids and
// two-phase flow"): the nonideal chemical potential and free energy of a node's
// density.  Host and device code, so that the same functions can be evaluated on
// the host.
#pragma once
#include <math.h>

namespace gblb {

// Equations of state, numbered as the lb_set_nonideal argument that selects them.
enum NiKind { kVdW = 1, kPengRobinson = 2, kCarnahanStarling = 3 };

struct NiEos {
    double a, b, theta0, kappa, eta;
    int kind;
};

// The same constants in the field type F, converted once on the host (an FP64-to-FP32 conversion
// in every thread runs at GB300's FP64 rate).
template <class F>
struct NiEosT {
    F a, b, theta0, kappa, eta;
    int kind;
};
template <class F>
inline NiEosT<F> ni_eos_in(const NiEos& e) {
    return NiEosT<F>{(F)e.a, (F)e.b, (F)e.theta0, (F)e.kappa, (F)e.eta, e.kind};
}

__host__ __device__ __forceinline__ double ni_log(double v) { return log(v); }
__host__ __device__ __forceinline__ float ni_log(float v) { return logf(v); }
__host__ __device__ __forceinline__ double ni_log1p(double v) { return log1p(v); }
__host__ __device__ __forceinline__ float ni_log1p(float v) { return log1pf(v); }

// Carnahan-Starling repulsion at packing fraction p = b rho / 4: its excess free energy per
// particle over theta0, f = (4p - 3p^2) / (1 - p)^2 (the integral of (Z - 1) / rho with
// Z = (1 + p + p^2 - p^3) / (1 - p)^3), and rho df/drho = p (4 - 2p) / (1 - p)^3.
template <class F>
__host__ __device__ __forceinline__ void cs_repulsion(F p, F& f, F& rdf) {
    const F inv = F(1) / (F(1) - p), inv2 = inv * inv;
    f = p * (F(4) - F(3) * p) * inv2;
    rdf = p * (F(4) - F(2) * p) * inv2 * inv;
}

// mu_nid and F_nid of node density r, in the field type F: the free energy without the
// ideal part theta0 rho (ln rho - 1), so that p = rho mu - F and both vanish as rho -> 0.
//   van der Waals       F = -theta0 rho ln(1 - b rho) - a rho^2
//   Peng-Robinson type  F = theta0 rho f - a rho L,  L = int_0^rho drho' / (1 + 2b rho' - b^2 rho'^2)
//                         = [ln(1 + (sqrt2 + 1) b rho) - ln(1 - (sqrt2 - 1) b rho)] / (2 sqrt2 b)
//   Carnahan-Starling   F = theta0 rho f - a rho^2
template <class F, class E>
__host__ __device__ __forceinline__ void ni_eos(F r, const E& e, F& mu, F& Fe) {
    const F th = F(e.theta0), a = F(e.a), br = F(e.b) * r;
    if (e.kind == kPengRobinson) {
        F f, rdf;
        cs_repulsion(F(0.25) * br, f, rdf);
        const F L = (ni_log1p(F(2.414213562373095) * br) - ni_log1p(F(-0.41421356237309503) * br)) *
                    F(0.35355339059327373) / F(e.b);
        Fe = r * th * f - a * r * L;
        mu = th * (f + rdf) - a * L - a * r / (F(1) + br * (F(2) - br));
    } else if (e.kind == kCarnahanStarling) {
        F f, rdf;
        cs_repulsion(F(0.25) * br, f, rdf);
        Fe = r * th * f - a * r * r;
        mu = th * (f + rdf) - F(2) * a * r;
    } else {
        const F L = ni_log(F(1) - br);
        Fe = -r * th * L - a * r * r;
        mu = -th * L + th * br / (F(1) - br) - F(2) * a * r;
    }
}

}  // namespace gblb
