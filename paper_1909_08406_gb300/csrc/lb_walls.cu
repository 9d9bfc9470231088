// Kinetic (diffuse) walls normal to z (Sec. "Viscous heat dissipation": the
// paper applies the kinetic boundary condition of Ansumali and Karlin 2002 at
// the walls and periodic conditions along them).
//
// Placement: in doubled coordinates the nodes occupy z2 = 2z + s in [0, 2 nz);
// the bottom wall lies at z2 = -1/2 and the top wall at z2 = 2 nz - 1/2, a
// quarter cell beyond the outermost node planes (channel height nz cells).
// Diffuse reflection: a post-collision population whose destination lies
// beyond a wall is absorbed by it; a population whose upwind position lies
// beyond a wall is emitted by it as rho_w f^eq_i(1, u_w, theta_w), the model's
// own equilibrium (linear in rho) at the wall's velocity and temperature, with
// rho_w the density that returns the absorbed mass (one value per wall and
// step, the balance taken over the whole wall plane).
//
// Per step, around the ordinary periodic step kernel (src -> dst):
//   k_wall_absorb   absorbed mass per wall, FP64, from src (partials per block)
//   k_wall_density  rho_w per wall and the 2 x 41 emitted working values
//   <periodic step> every node; nodes next to a wall pull wrapped values here
//   k_step_walls    recomputes the nodes of the 2 outermost cell layers at
//                   each wall (the only ones with upwind positions beyond a
//                   wall: links reach 2 cells), src -> dst, overwriting them.
// The sums are taken in a fixed order, so a step is deterministic.
#include <math.h>

#include "lb_ctx.h"
#include "lb_kernels.cuh"

namespace gblb {

constexpr int kWallBlocks = 64;     // absorb partials per wall
constexpr int kWallThreads = 256;

// Device block of one context's walls (doubles unless noted):
//   e[2][kQ]        f^eq_i(1, u_w, theta_w) of the bottom and top wall
//   emit[2]         sum over the (node, i) pairs a unit-density wall feeds
//   part[2][kWallBlocks]  absorbed-mass partials
//   rho[2]          rho_w of the last step
//   vd[2][kQ]       emitted working values (FP64 codec)
//   vf[2][kQ]       emitted working values as float (FP32 arithmetic codecs)
struct WallLayout {
    static constexpr int e = 0;
    static constexpr int emit = e + 2 * kQ;
    static constexpr int part = emit + 2;
    static constexpr int rho = part + 2 * kWallBlocks;
    static constexpr int vd = rho + 2;
    static constexpr int vf = vd + 2 * kQ;  // float[2 * kQ] from here
    static constexpr int doubles = vf + kQ;  // 2 * kQ floats fit in kQ doubles
};

// f^eq_i(1, u_w, theta_w) of both walls and the unit emission sums, in FP64.
// wall[8] = {u_x, u_y, u_z, theta} of the bottom wall, then of the top wall.
template <int EQ>
__global__ void k_wall_setup(double* __restrict__ blk, Dims d, Consts<double> K, double theta0, double wx0,
                             double wy0, double wz0, double t0, double w1x, double w1y, double w1z, double t1) {
    if (threadIdx.x >= 2) return;
    const int side = threadIdx.x;
    NodeState<double> st;
    st.drho = 0.0;
    st.rho = 1.0;
    st.ux = side ? w1x : wx0;
    st.uy = side ? w1y : wy0;
    st.uz = side ? w1z : wz0;
    st.eta = (side ? t1 : t0) / theta0 - 1.0;
    double zero[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) zero[i] = 0.0;
    double* e = blk + WallLayout::e + side * kQ;
    bool ok = true;
    equilibrium_relax<CodecF64, EQ>(st, K, 1.0, 0.0, zero, [&](auto I, double val) { e[I] = val; }, ok);
    // a unit-density wall feeds population i (c_iz > 0 for the bottom, < 0 for the top) into
    // the node planes z2 with z2 - 2 c_iz beyond it: |2 c_iz| planes of nx * ny nodes
    double sum = 0.0;
    for (int i = 0; i < kQ; ++i) {
        const int cz = c_vel.v[i].z;
        const int planes = side ? (cz < 0 ? -cz : 0) : (cz > 0 ? cz : 0);
        sum += (double)planes * e[i];
    }
    blk[WallLayout::emit + side] = sum * (double)d.nx * (double)d.ny;
    blk[WallLayout::rho + side] = ok ? 1.0 : nan("");
}

// Absorbed mass: sum of f over the populations of the two outermost cell layers at the wall
// whose destination z2 + 2 c_iz lies beyond it.  blockIdx.y: 0 bottom, 1 top.
template <class Codec>
__global__ void __launch_bounds__(kWallThreads) k_wall_absorb(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                              Consts<double> K, double* __restrict__ blk) {
    const int side = blockIdx.y;
    const int64_t nxy = (int64_t)d.nx * d.ny;
    const int64_t items = 4 * nxy;  // (layer, s) x (y, x)
    const int64_t nz2 = 2 * (int64_t)d.nz;
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < items;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int ls = (int)(k / nxy);
        const int64_t xy = k - ls * nxy;
        const int layer = ls >> 1, s = ls & 1;
        const int z = side ? d.nz - 2 + layer : layer;
        const int64_t z2 = 2 * (int64_t)z + s;
        const typename Codec::raw_t* p = src + ((int64_t)s * kQ * d.plane + (int64_t)z * nxy + xy);
        static_for<kQ>([&](auto I) {
            constexpr Vel c = vel(I);
            if constexpr (c.z != 0) {
                const int64_t dest = z2 + c.z;
                if (side ? dest >= nz2 : dest < 0) {
                    const double v = (double)Codec::value(p[(int64_t)I * d.plane]);
                    const double w = K.w[c.shell];
                    acc += Codec::stores_f ? v : w * (1.0 + v * (1.0 / Codec::kScale));
                }
            }
        });
    }
    __shared__ double red[kWallThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kWallThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) blk[WallLayout::part + side * kWallBlocks + blockIdx.x] = red[0];
}

// rho_w = absorbed / emitted-at-unit-density per wall, and the working values the wall
// emits: f for the FP64 codec, (f / w - 1) * scale for the deviation codecs.
template <class Codec>
__global__ void k_wall_density(double* __restrict__ blk, Consts<double> K) {
    __shared__ double rho[2];
    if (threadIdx.x < 2) {
        double a = 0.0;
        for (int b = 0; b < kWallBlocks; ++b) a += blk[WallLayout::part + threadIdx.x * kWallBlocks + b];
        rho[threadIdx.x] = a / blk[WallLayout::emit + threadIdx.x];
        blk[WallLayout::rho + threadIdx.x] = rho[threadIdx.x];
    }
    __syncthreads();
    float* vf = reinterpret_cast<float*>(blk + WallLayout::vf);
    for (int k = threadIdx.x; k < 2 * kQ; k += blockDim.x) {
        const int side = k / kQ, i = k - side * kQ;
        const double e = blk[WallLayout::e + k];
        const double w = K.w[c_vel.v[i].shell];
        const double r = rho[side];
        // deviation of rho_w e_i from the rest weight: (r - 1) + r (e / w - 1)
        const double v = Codec::stores_f ? r * e : ((r - 1.0) + r * (e / w - 1.0)) * Codec::kScale;
        blk[WallLayout::vd + k] = v;
        vf[k] = (float)v;
    }
}

// The update of the nodes in the two outermost cell layers at each wall: the gather of
// step_node with every upwind position beyond a wall replaced by that wall's emission.
// Grid: x = x chunks, y = (layer 0..3, s, y) rows; layers 0, 1 at the bottom, 2, 3 at the top.
template <class Codec, int EQ>
__global__ void __launch_bounds__(kStepThreads) k_step_walls(const typename Codec::raw_t* __restrict__ src,
                                                             typename Codec::raw_t* __restrict__ dst, Dims d,
                                                             Consts<typename Codec::R> K, typename Codec::R tb,
                                                             const typename Codec::R* __restrict__ vwall,
                                                             int* __restrict__ err) {
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

    R v[kQ];
    static_for<kQ>([&](auto I) {
        constexpr Vel c = vel(I);
        const int up = z2 - c.z;  // doubled z of the upwind position
        if (up < 0) {
            v[I] = vwall[I];
        } else if (up >= nz2) {
            v[I] = vwall[kQ + I];
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

cudaError_t launch_wall_setup(int eq, double* blk, const Dims& d, const LaunchConsts& c, const double wall[8],
                              cudaStream_t st) {
    return with_eq(eq, [&](auto E) {
        k_wall_setup<decltype(E)::value><<<1, 32, 0, st>>>(blk, d, c.kd, c.theta0, wall[0], wall[1], wall[2], wall[3],
                                                           wall[4], wall[5], wall[6], wall[7]);
        return cudaGetLastError();
    });
}

cudaError_t launch_wall_step(int prec, int eq, int variant, const void* src, void* dst, const Dims& d,
                             const LaunchConsts& c, double twobeta, double* blk, int* err, cudaStream_t st) {
    cudaError_t e = with_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        k_wall_absorb<C><<<dim3(kWallBlocks, 2), kWallThreads, 0, st>>>(static_cast<const typename C::raw_t*>(src),
                                                                         d, c.kd, blk);
        k_wall_density<C><<<1, 96, 0, st>>>(blk, c.kd);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    e = launch_step(prec, eq, variant, src, dst, d, c, twobeta, err, st);
    if (e != cudaSuccess) return e;
    return with_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        using R = typename C::R;
        const int th = step_threads(d);
        const dim3 grid((unsigned)((d.nx + th - 1) / th), (unsigned)(8 * d.ny));
        const R* vw;
        if constexpr (sizeof(R) == 8)
            vw = reinterpret_cast<const R*>(blk + WallLayout::vd);
        else
            vw = reinterpret_cast<const R*>(blk + WallLayout::vf);
        const Consts<R>* K;
        if constexpr (sizeof(R) == 8)
            K = &c.kd;
        else
            K = &c.kf;
        return with_eq(eq, [&](auto E) {
            k_step_walls<C, decltype(E)::value><<<grid, th, 0, st>>>(
                static_cast<const typename C::raw_t*>(src), static_cast<typename C::raw_t*>(dst), d, *K,
                (R)twobeta, vw, err);
            return cudaGetLastError();
        });
    });
}

size_t wall_block_bytes() { return sizeof(double) * WallLayout::doubles; }
int wall_rho_offset() { return WallLayout::rho; }

}  // namespace gblb
