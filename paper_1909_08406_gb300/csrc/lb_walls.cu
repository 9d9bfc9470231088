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
//   k_wall_density  rho_w per wall from the absorbed-mass partials, and the
//                   2 x 41 emitted working values
//   <periodic step> every node; nodes next to a wall pull wrapped values here
//   k_step_walls    recomputes the nodes of the 2 outermost cell layers at
//                   each wall (the only ones with upwind positions beyond a
//                   wall: links reach 2 cells), src -> dst, overwriting them,
//                   and sums, per block, the mass that the next step's walls
//                   absorb from what it stores (those layers are the only
//                   ones with populations leaving through a wall).
// After the state is set from outside (fields, populations, a checkpoint,
// new walls), k_wall_absorb forms the same partials from the stored state once.
// Every sum is taken in a fixed order, so a step is deterministic.
#include <math.h>

#include "lb_ctx.h"
#include "lb_kernels.cuh"

namespace gblb {

constexpr int kDensityThreads = 512;

// Device block of one context's walls (doubles unless noted):
//   e[2][kQ]        f^eq_i(1, u_w, theta_w) of the bottom and top wall
//   emit[2]         sum over the (node, i) pairs a unit-density wall feeds
//   wsum[2]         sum of w_i over the (node, i) pairs a wall absorbs: the rest-state part of
//                   the absorbed mass, which the deviation codecs do not sum per node
//   rho[2]          rho_w of the last step
//   vd[2][kQ]       emitted working values (FP64 codec)
//   vf[2][kQ]       emitted working values as float (FP32 arithmetic codecs)
struct WallLayout {
    static constexpr int e = 0;
    static constexpr int emit = e + 2 * kQ;
    static constexpr int wsum = emit + 2;
    static constexpr int rho = wsum + 2;
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
    // and absorbs population i (c_iz < 0 at the bottom, > 0 at the top) from |2 c_iz| planes
    double sum = 0.0, wsum = 0.0;
    for (int i = 0; i < kQ; ++i) {
        const int cz = c_vel.v[i].z;
        const int planes = side ? (cz < 0 ? -cz : 0) : (cz > 0 ? cz : 0);
        const int out_planes = side ? (cz > 0 ? cz : 0) : (cz < 0 ? -cz : 0);
        sum += (double)planes * e[i];
        wsum += (double)out_planes * K.w[c_vel.v[i].shell];
    }
    blk[WallLayout::emit + side] = sum * (double)d.nx * (double)d.ny;
    blk[WallLayout::wsum + side] = wsum * (double)d.nx * (double)d.ny;
    blk[WallLayout::rho + side] = ok ? 1.0 : nan("");
}

// Block sum in a fixed order (warp trees, then the warps' sums in order); every thread of
// the block must call it.  The result is valid in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v) {
    __shared__ double warp_sums[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sums[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) t += warp_sums[k];
    return t;
}

// Absorbed mass of the stored state, in the partial layout and summation order of
// k_step_walls (one partial per block of its grid, each node's populations in index order,
// block_sum_fixed), so that a state set from outside gives the same wall densities as the
// same state reached by stepping.
// A stored value's share of the absorbed mass: f itself for the FP64 codec; for the deviation
// codecs w h (the rest-state part w is added once per wall, from wsum), in the compute type.
template <class Codec>
__device__ __forceinline__ typename Codec::R absorbed_part(typename Codec::R v, typename Codec::R w) {
    using R = typename Codec::R;
    if constexpr (Codec::stores_f)
        return v;
    else
        return w * (v * R(1.0 / Codec::kScale));
}

template <class Codec>
__global__ void __launch_bounds__(kStepThreads) k_wall_absorb(const typename Codec::raw_t* __restrict__ src, Dims d,
                                                              Consts<typename Codec::R> K,
                                                              double* __restrict__ part) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (x < d.nx) {
        const int row = blockIdx.y;  // (layer * 2 + s) * ny + y
        const int y = row % d.ny;
        const int ls = row / d.ny;
        const int layer = ls >> 1, s = ls & 1;
        const int z = layer < 2 ? layer : d.nz - 4 + layer;
        const int z2 = 2 * z + s, nz2 = 2 * d.nz;
        const bool bottom = layer < 2;
        const typename Codec::raw_t* p =
            src + ((int64_t)s * kQ * d.plane + ((int64_t)z * d.ny + y) * d.nx + x);
        typename Codec::R a = 0;
        static_for<kQ>([&](auto I) {
            constexpr Vel c = vel(I);
            if constexpr (c.z != 0) {
                const int dest = z2 + c.z;
                if (bottom ? dest < 0 : dest >= nz2)
                    a += absorbed_part<Codec>(Codec::value(p[(int64_t)I * d.plane]), K.w[c.shell]);
            }
        });
        acc = (double)a;
    }
    const double t = block_sum_fixed(acc);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// part[side * nper + k], k < nper: the absorbed-mass partials of each wall.
template <class Codec>
__global__ void __launch_bounds__(kDensityThreads) k_wall_density(double* __restrict__ blk, Consts<double> K,
                                                                  const double* __restrict__ part, int nper) {
    __shared__ double red[2][kDensityThreads];
    __shared__ double rho[2];
    for (int side = 0; side < 2; ++side) {
        double a = 0.0;
        for (int k = threadIdx.x; k < nper; k += kDensityThreads) a += part[side * nper + k];
        red[side][threadIdx.x] = a;
    }
    __syncthreads();
    for (int h = kDensityThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) {
        const double absorbed = red[threadIdx.x][0] + (Codec::stores_f ? 0.0 : blk[WallLayout::wsum + threadIdx.x]);
        rho[threadIdx.x] = absorbed / blk[WallLayout::emit + threadIdx.x];
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


// One node of k_step_walls; returns the mass its stored values send through the wall.
template <class Codec, int EQ>
__device__ __forceinline__ double wall_node(const typename Codec::raw_t* __restrict__ src,
                                            typename Codec::raw_t* __restrict__ dst, const Dims& d,
                                            const Consts<typename Codec::R>& K, typename Codec::R tb,
                                            const typename Codec::R* __restrict__ vwall, int* __restrict__ err,
                                            int x) {
    using R = typename Codec::R;
    using T = typename Codec::raw_t;
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
    R absorbed = 0;
    const bool bottom = layer < 2;
    equilibrium_relax<Codec, EQ>(st, K, tb * R(Codec::kScale), R(1) - tb, v,
                                 [&](auto I, R val) {
                                     const T raw = Codec::to_raw(val);
                                     out[(int64_t)I * d.plane] = raw;
                                     constexpr Vel c = vel(I);
                                     if constexpr (c.z != 0) {
                                         const int dest = z2 + c.z;
                                         if (bottom ? dest < 0 : dest >= nz2)
                                             absorbed += absorbed_part<Codec>(Codec::value(raw), K.w[c.shell]);
                                     }
                                 },
                                 ok);
    if (!ok) atomicOr(err, 1);
    return (double)absorbed;
}

// The update of the nodes in the two outermost cell layers at each wall: the gather of
// step_node with every upwind position beyond a wall replaced by that wall's emission.
// Grid: x = x chunks, y = (layer 0..3, s, y) rows; layers 0, 1 at the bottom, 2, 3 at the top.
// part[blockIdx.y * gridDim.x + blockIdx.x] receives the mass that the stored values will
// send through the block's wall in the next step (bottom partials first, then top).
template <class Codec, int EQ>
__global__ void __launch_bounds__(kStepThreads) k_step_walls(const typename Codec::raw_t* __restrict__ src,
                                                             typename Codec::raw_t* __restrict__ dst, Dims d,
                                                             Consts<typename Codec::R> K, typename Codec::R tb,
                                                             const typename Codec::R* __restrict__ vwall,
                                                             double* __restrict__ part, int* __restrict__ err) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double absorbed = 0.0;
    if (x < d.nx) absorbed = wall_node<Codec, EQ>(src, dst, d, K, tb, vwall, err, x);
    const double t = block_sum_fixed(absorbed);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
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

// Blocks of k_step_walls along x for this grid (and the step kernels' row width).
static int wall_chunks(const Dims& d) {
    const int th = step_threads(d);
    return (d.nx + th - 1) / th;
}

size_t wall_part_doubles(const Dims& d) { return (size_t)8 * d.ny * wall_chunks(d); }

cudaError_t launch_wall_step(int prec, int eq, int variant, const void* src, void* dst, const Dims& d,
                             const LaunchConsts& c, double twobeta, double* blk, double* part, bool sums_valid,
                             int* err, cudaStream_t st) {
    const int chunks = wall_chunks(d);
    cudaError_t e = with_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        using R = typename C::R;
        const int nper = 4 * d.ny * chunks;  // partials per wall (k_step_walls' blocks)
        const Consts<R>* K;
        if constexpr (sizeof(R) == 8)
            K = &c.kd;
        else
            K = &c.kf;
        if (!sums_valid)
            k_wall_absorb<C><<<dim3((unsigned)chunks, (unsigned)(8 * d.ny)), step_threads(d), 0, st>>>(
                static_cast<const typename C::raw_t*>(src), d, *K, part);
        k_wall_density<C><<<1, kDensityThreads, 0, st>>>(blk, c.kd, part, nper);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    e = launch_step(prec, eq, variant, src, dst, d, c, twobeta, err, st);
    if (e != cudaSuccess) return e;
    return with_codec(prec, [&](auto codec) {
        using C = decltype(codec);
        using R = typename C::R;
        const int th = step_threads(d);
        const dim3 grid((unsigned)chunks, (unsigned)(8 * d.ny));
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
                (R)twobeta, vw, part, err);
            return cudaGetLastError();
        });
    });
}

size_t wall_block_bytes() { return sizeof(double) * WallLayout::doubles; }
int wall_rho_offset() { return WallLayout::rho; }

}  // namespace gblb
