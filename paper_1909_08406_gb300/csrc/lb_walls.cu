// Kinetic (diffuse) walls normal to z (Sec. "Viscous heat dissipation": the
// paper applies the kinetic boundary condition of Ansumali and Karlin 2002 at
// the walls and periodic conditions along them).
//
// Placement: in doubled coordinates the nodes occupy z2 = 2z + s in [0, 2 nz);
// the bottom wall lies at z2 = -1/2 and the top wall at z2 = 2 nz - 1/2, a
// quarter cell beyond the outermost node planes (channel height nz cells).
// Each wall is cut into the cell columns (x, y) of the grid: the bottom wall's
// column x holds the doubled lateral positions {2x, 2x + 1}, the top wall's
// {2x - 1, 2x} (the walls face the A and the B outermost plane, and the
// half-cell-shifted mirror that exchanges the walls carries one partition onto
// the other).  Diffuse reflection, column by column: a post-collision
// population whose destination lies beyond a wall is absorbed by the column
// that contains the destination; a population whose upwind position lies
// beyond a wall is emitted by the column that contains that position, as
// rho_w f^eq_i(1, u_w, theta_w), the model's own equilibrium (linear in rho)
// at the column's velocity and temperature, with rho_w the density that
// returns the column's absorbed mass.
//
// Per step, around the ordinary periodic step kernel (src -> dst):
//   k_wall_columns  absorbed mass and rho_w of every wall column, gathered
//                   from src in a fixed order
//   <periodic step> every node; nodes next to a wall pull wrapped values here
//   k_step_walls    recomputes the nodes of the 2 outermost cell layers at
//                   each wall (the only ones with upwind positions beyond a
//                   wall: links reach 2 cells), src -> dst, overwriting them.
#include <math.h>

#include "lb_ctx.h"
#include "lb_kernels.cuh"

namespace gblb {

// floor(v / 2) for the small integers of the column arithmetic (v >= -8)
__host__ __device__ __forceinline__ int half_floor(int v) { return (v + 8) / 2 - 4; }

// Node planes (doubled z) next to a wall from beyond which population i arrives (in) or
// through which it leaves (out): |2 c_iz| of them when c_iz points the right way, else 0.
__host__ __device__ __forceinline__ int planes_in(int cz, int side) { return side ? (cz < 0 ? -cz : 0) : (cz > 0 ? cz : 0); }
__host__ __device__ __forceinline__ int planes_out(int cz, int side) { return side ? (cz > 0 ? cz : 0) : (cz < 0 ? -cz : 0); }

// The walls' device data (one allocation; R is the compute type of the storage codec):
//   param[2][3][ncol]  u_x, u_y, theta of every column (double)
//   emit[2][ncol]      sum_i planes_in_i e_i of the column: what it emits at unit density
//   rho[2][ncol]       rho_w of every column in the last step (double)
//   wsum[2]            sum_i planes_out_i w_i: the rest-state part of a column's absorbed mass,
//                      which the deviation codecs do not sum per population
//   e[2][kQ][ncol]     e_i = f^eq_i(1, u_w, theta_w) (FP64 codec) or e_i / w_i - 1 (deviation
//                      codecs), in R
//   dr[2][ncol]        rho_w (FP64 codec) or rho_w - 1 (deviation codecs), in R
//   bad                set by the set-up if a column has no equilibrium
struct WallPtrs {
    double *param, *emit, *rho, *wsum;
    void *e, *dr;
    int* bad;
};

static size_t round16(size_t b) { return (b + 15) / 16 * 16; }

static WallPtrs wall_ptrs(void* blk, int64_t ncol, size_t rsize) {
    char* p = static_cast<char*>(blk);
    WallPtrs w;
    w.param = reinterpret_cast<double*>(p);
    w.emit = w.param + 6 * ncol;
    w.rho = w.emit + 2 * ncol;
    w.wsum = w.rho + 2 * ncol;
    size_t off = sizeof(double) * (size_t)(10 * ncol + 2);
    off = round16(off);
    w.e = p + off;
    off += round16((size_t)(2 * kQ * ncol) * rsize);
    w.dr = p + off;
    off += round16((size_t)(2 * ncol) * rsize);
    w.bad = reinterpret_cast<int*>(p + off);
    return w;
}

static size_t rsize_of(int prec) { return prec == kF64 ? 8 : 4; }

size_t wall_block_bytes(int64_t ncol, int prec) {
    const size_t rs = rsize_of(prec);
    return round16(sizeof(double) * (size_t)(10 * ncol + 2)) + round16((size_t)(2 * kQ * ncol) * rs) +
           round16((size_t)(2 * ncol) * rs) + 16;
}

double* wall_params(void* blk) { return static_cast<double*>(blk); }
double* wall_rho(void* blk, int64_t ncol) { return static_cast<double*>(blk) + 8 * ncol; }
int* wall_bad_flag(void* blk, int64_t ncol, int prec) { return wall_ptrs(blk, ncol, rsize_of(prec)).bad; }

// Per column: f^eq(1, u_w, theta_w) in FP64, its unit emission, and the codec's copy of it.
template <class Codec, int EQ>
__global__ void k_wall_setup(WallPtrs w, Dims d, Consts<double> K, double theta0) {
    using R = typename Codec::R;
    const int64_t ncol = (int64_t)d.nx * d.ny;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * ncol) return;
    const int side = (int)(k / ncol);
    const int64_t col = k - side * ncol;
    const double* pr = w.param + side * 3 * ncol;
    NodeState<double> st;
    st.drho = 0.0;
    st.rho = 1.0;
    st.ux = pr[col];
    st.uy = pr[ncol + col];
    st.uz = 0.0;
    st.eta = pr[2 * ncol + col] / theta0 - 1.0;
    double zero[kQ], e[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) zero[i] = 0.0;
    bool ok = state_ok(st);
    equilibrium_relax<CodecF64, EQ>(st, K, 1.0, 0.0, zero, [&](auto I, double val) { e[I] = val; }, ok);
    double emit = 0.0;
    R* ec = static_cast<R*>(w.e) + (int64_t)side * kQ * ncol + col;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        emit += (double)planes_in(c_vel.v[i].z, side) * e[i];
        const double wi = K.w[c_vel.v[i].shell];
        ec[(int64_t)i * ncol] = (R)(Codec::stores_f ? e[i] : e[i] / wi - 1.0);
        ok = ok && isfinite(e[i]) && e[i] > 0.0;
    }
    w.emit[k] = emit;
    w.rho[k] = 1.0;
    static_cast<R*>(w.dr)[k] = (R)(Codec::stores_f ? 1.0 : 0.0);
    if (col == 0) {
        double ws = 0.0;
        for (int i = 0; i < kQ; ++i) ws += (double)planes_out(c_vel.v[i].z, side) * K.w[c_vel.v[i].shell];
        w.wsum[side] = ws;
    }
    if (!ok) atomicOr(w.bad, 1);
}

// Absorbed mass and rho_w of every wall column.  Column (cx, cy) of a wall absorbs population
// i from the node planes z2 it leaves through the wall, from the source cell whose destination
// falls in the column: x = cx - floor((s + 2 c_ix + side) / 2), likewise y.  The sum runs in a
// fixed order (population, then plane), so a step is deterministic and a state set from outside
// gives the same densities as the same state reached by stepping.
template <class Codec>
__global__ void __launch_bounds__(128) k_wall_columns(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                      Consts<typename Codec::R> K, WallPtrs w) {
    using R = typename Codec::R;
    const int64_t ncol = (int64_t)d.nx * d.ny;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * ncol) return;
    const int side = (int)(k / ncol);
    const int64_t col = k - side * ncol;
    const int cy = (int)(col / d.nx), cx = (int)(col - (int64_t)cy * d.nx);
    const int nz2 = 2 * d.nz;
    R acc = 0;
    static_for<kQ>([&](auto I) {
        constexpr Vel c = vel(I);
        if constexpr (c.z != 0) {
            const int np = planes_out(c.z, side);
            for (int j = 0; j < np; ++j) {
                const int z2 = side ? nz2 - np + j : j;
                const int s = z2 & 1, z = z2 >> 1;
                int x = cx - half_floor(s + c.x + side), y = cy - half_floor(s + c.y + side);
                x = x < 0 ? x + d.nx : (x >= d.nx ? x - d.nx : x);
                y = y < 0 ? y + d.ny : (y >= d.ny ? y - d.ny : y);
                const R v =
                    Codec::value(src[((int64_t)s * kQ + I) * d.plane + ((int64_t)z * d.ny + y) * d.nx + x]);
                if constexpr (Codec::stores_f)
                    acc += v;
                else
                    acc += K.w[c.shell] * (v * R(1.0 / Codec::kScale));
            }
        }
    });
    const double absorbed = (double)acc + (Codec::stores_f ? 0.0 : w.wsum[side]);
    const double rho = absorbed / w.emit[k];
    w.rho[k] = rho;
    static_cast<R*>(w.dr)[k] = (R)(Codec::stores_f ? rho : rho - 1.0);
}

// The update of the nodes in the two outermost cell layers at each wall: the gather of
// step_node with every upwind position beyond a wall replaced by the emission of the wall
// column that contains it.  Grid: x = x chunks, y = (layer 0..3, s, y) rows; layers 0, 1 at the
// bottom, 2, 3 at the top.
template <class Codec, int EQ>
__global__ void __launch_bounds__(kStepThreads) k_step_walls(const typename Codec::raw_t* __restrict__ src,
                                                             typename Codec::raw_t* __restrict__ dst, Dims d,
                                                             Consts<typename Codec::R> K, typename Codec::R tb,
                                                             WallPtrs w, int* __restrict__ err) {
    using R = typename Codec::R;
    using T = typename Codec::raw_t;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= d.nx) return;
    const int row = blockIdx.y;  // (layer * 2 + s) * ny + y
    const int y = row % d.ny;
    const int ls = row / d.ny;
    const int layer = ls >> 1, s = ls & 1;
    const int z = layer < 2 ? layer : d.nz - 4 + layer;
    const int z2 = 2 * z + s, nz2 = 2 * d.nz;
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
    const R* we = static_cast<const R*>(w.e);
    const R* wdr = static_cast<const R*>(w.dr);

    R v[kQ];
    static_for<kQ>([&](auto I) {
        constexpr Vel c = vel(I);
        const int up = z2 - c.z;  // doubled z of the upwind position
        if (up < 0 || up >= nz2) {
            const int side = up < 0 ? 0 : 1;
            // the wall column containing the upwind position's (x, y)
            int cx = x + half_floor(s - c.x + side), cy = y + half_floor(s - c.y + side);
            cx = cx < 0 ? cx + d.nx : (cx >= d.nx ? cx - d.nx : cx);
            cy = cy < 0 ? cy + d.ny : (cy >= d.ny ? cy - d.ny : cy);
            const int64_t col = (int64_t)cy * d.nx + cx;
            const R e = we[((int64_t)side * kQ + I) * nxy + col];
            const R r = wdr[side * nxy + col];
            if constexpr (Codec::stores_f)
                v[I] = r * e;
            else  // (rho_w e_i / w_i - 1) scaled: dr + he + dr he
                v[I] = (r + e + r * e) * R(Codec::kScale);
        } else if constexpr (c.shell == 5) {
            const int64_t off = (c.z > 0 ? hzp : hzm) + (c.y > 0 ? hyp : hym) + (c.x > 0 ? hxp : hxm);
            v[I] = Codec::value(other[(int64_t)I * d.plane + off]);
        } else {
            const int64_t off = zo[c.z / 2 + 2] + yo[c.y / 2 + 2] + xs[c.x / 2 + 2];
            v[I] = Codec::value(same[(int64_t)I * d.plane + off]);
        }
    });

    R dv[kQ];
    constexpr R inv_scale = R(1.0 / Codec::kScale);
    static_for<kQ>([&](auto I) { dv[I] = Codec::dev(v[I], K.w[vel(I).shell] * inv_scale); });
    const NodeState<R> st = state_from_moments(moments_from_dev(dv), K);
    bool ok = state_ok(st);
    T* out = dst + (int64_t)s * kQ * d.plane + (int64_t)z * nxy + (int64_t)y * d.nx + x;
    equilibrium_relax<Codec, EQ>(st, K, tb * R(Codec::kScale), R(1) - tb, v,
                                 [&](auto I, R val) { out[(int64_t)I * d.plane] = Codec::to_raw(val); }, ok);
    if (!ok) atomicOr(err, 1);
}

template <class F>
static cudaError_t with_codec(int prec, F&& f) {
    switch (prec) {
        case kF64: return f(CodecF64{});
        case kF32: return f(CodecF32{});
        case kF16: return f(CodecF16{});
        case kBF16: return f(CodecBF16{});
        default: return cudaErrorInvalidValue;
    }
}

template <class F>
static cudaError_t with_eq(int eq, F&& f) {
    switch (eq) {
        case 0: return f(std::integral_constant<int, 0>{});
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        default: return cudaErrorInvalidValue;
    }
}

template <class C>
static const Consts<typename C::R>& consts_for(const LaunchConsts& c) {
    if constexpr (sizeof(typename C::R) == 8)
        return c.kd;
    else
        return c.kf;
}

cudaError_t launch_wall_setup(int prec, int eq, void* blk, const Dims& d, const LaunchConsts& c, cudaStream_t st) {
    const int64_t ncol = (int64_t)d.nx * d.ny;
    return with_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        const WallPtrs w = wall_ptrs(blk, ncol, sizeof(typename C::R));
        cudaError_t e = cudaMemsetAsync(w.bad, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        return with_eq(eq, [&](auto E) {
            k_wall_setup<C, decltype(E)::value><<<(unsigned)((2 * ncol + 127) / 128), 128, 0, st>>>(w, d, c.kd,
                                                                                                  c.theta0);
            return cudaGetLastError();
        });
    });
}

cudaError_t launch_wall_step(int prec, int eq, int variant, const void* src, void* dst, const Dims& d,
                             const LaunchConsts& c, double twobeta, void* blk, int* err, cudaStream_t st) {
    const int64_t ncol = (int64_t)d.nx * d.ny;
    cudaError_t e = with_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        const WallPtrs w = wall_ptrs(blk, ncol, sizeof(typename C::R));
        k_wall_columns<C><<<(unsigned)((2 * ncol + 127) / 128), 128, 0, st>>>(
            static_cast<const typename C::raw_t*>(src), d, consts_for<C>(c), w);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    e = launch_step(prec, eq, variant, src, dst, d, c, twobeta, err, st);
    if (e != cudaSuccess) return e;
    return with_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        using R = typename C::R;
        const WallPtrs w = wall_ptrs(blk, ncol, sizeof(R));
        const int th = step_threads(d);
        const dim3 grid((unsigned)((d.nx + th - 1) / th), (unsigned)(8 * d.ny));
        return with_eq(eq, [&](auto E) {
            k_step_walls<C, decltype(E)::value><<<grid, th, 0, st>>>(
                static_cast<const typename C::raw_t*>(src), static_cast<typename C::raw_t*>(dst), d,
                consts_for<C>(c), (R)twobeta, w, err);
            return cudaGetLastError();
        });
    });
}

}  // namespace gblb
