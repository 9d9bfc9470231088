// Host-side launchers of the RD3Q41 kernels (one set per storage precision).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lb_common.cuh"

namespace gblb {

struct W41 {
    double w[kQ];  // per-population weights, library order
};

struct LaunchConsts {
    Consts<float> kf;
    Consts<double> kd;
    W41 w41;
    double theta0;
};

// Storage precision codes (match lb_precision in gblb.h).
enum Prec { kF64 = 0, kF32 = 1, kF16 = 2, kBF16 = 3 };

// Step kernels (values match LB_KERNEL_* in gblb.h).
enum StepKernel {
    kKernelAuto = -1,
    kKernelDirect1 = 0,
    kKernelDirect2 = 1,
    kKernelDirect2R = 2,
    kKernelStaged = 3,
    kKernelWarpSpec = 4,
    kKernelDirect2X = 5,
    kKernelDirect2XL = 6
};

// The kernel a request resolves to for this precision and grid (falls back where one does not apply).
int resolve_kernel(int prec, const Dims& d, int kernel);

// Tile width of the staged kernel for this grid and precision, 0 if it does not apply.
int tma_tile_width(int prec, const Dims& d);

size_t storage_bytes(int prec);

// One fused pull step src -> dst over the whole grid.
cudaError_t launch_step(int prec, int eq, int variant, const void* src, void* dst, const Dims& d,
                        const LaunchConsts& c, double twobeta, int* err, cudaStream_t st);

// One fused step with the stochastic BF16 store (BF16 storage, series equilibrium with the
// momentum projection, periodic grid); sr_key is the step key k_t of lb_common.cuh.
cudaError_t launch_step_sr(const void* src, void* dst, const Dims& d, const LaunchConsts& c, double twobeta, int* err,
                           cudaStream_t st, uint32_t sr_key);

// Equilibrium of float64 fields for nodes [q0, q0 + count).
cudaError_t launch_init(int prec, int eq, void* dst, const Dims& d, const LaunchConsts& c, int64_t q0,
                        int64_t count, const double* rho, const double* u, int64_t ustride, const double* theta,
                        int* err, cudaStream_t st);

// Node moments for nodes [q0, q0 + count) into float64 fields (any may be null).
cudaError_t launch_moments(int prec, const void* src, const Dims& d, const LaunchConsts& c, int64_t q0, int64_t count,
                           double* rho, double* u, int64_t ustride, double* theta, cudaStream_t st);

// Global FP64 sums (drho, jx, jy, jz, dk) -> out5 (device), via nblocks partials.
cudaError_t launch_conserved(int prec, const void* src, const Dims& d, const LaunchConsts& c, double* partials,
                             int nblocks, double* out5, cudaStream_t st, int64_t z0 = 0, int64_t nzr = -1);

// Halo planes of a z slab: copy, for each of n (plane, population) entries, both sub-lattices' ny nx
// elements of that population on that plane between the population array and a packed buffer
// [entry][s][y][x] (pack: array -> buffer; else buffer -> array).
struct HaloList {
    int n;
    int plane[2 * kQ];
    int pop[2 * kQ];
};
cudaError_t launch_halo_copy(int prec, void* f, const Dims& d, const HaloList& list, void* buf, bool pack,
                             cudaStream_t st);

// Raw storage <-> float64 populations for elements [e0, e0 + count).
cudaError_t launch_to_f64(int prec, const void* src, const Dims& d, const LaunchConsts& c, int64_t e0, int64_t count,
                          double* f, cudaStream_t st);
cudaError_t launch_from_f64(int prec, const double* f, void* dst, const Dims& d, const LaunchConsts& c, int64_t e0,
                            int64_t count, cudaStream_t st);

// Per-precision step launchers (defined in the per-precision translation units).
cudaError_t launch_step_f64(int eq, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                            double twobeta, int* err, cudaStream_t st);
cudaError_t launch_step_f32(int prec, bool project, int variant, const void* src, void* dst, const Dims& d,
                            const LaunchConsts& c, double twobeta, int* err, cudaStream_t st);
// The exact-entropic-equilibrium update (FP32 arithmetic, any storage but FP64), k_step only.
cudaError_t launch_step_entropic(int prec, int eq, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                                 double twobeta, int* err, cudaStream_t st);

// Kinetic walls normal to z (lb_walls.cu), one device block per context of
// wall_block_bytes(nx * ny, prec): per-column parameters (wall_params: [2][3][ny][nx] doubles,
// u_x, u_y, theta of the bottom then the top wall's cell columns), the columns' rho_w of the
// last step (wall_rho: [2][ny][nx] doubles) and the derived data of lb_walls.cu.
size_t wall_block_bytes(int64_t ncol, int prec);
double* wall_params(void* blk);
double* wall_rho(void* blk, int64_t ncol);
int* wall_bad_flag(void* blk, int64_t ncol, int prec);
// Derive the columns' equilibria from the parameters (sets the bad flag if one has none).
cudaError_t launch_wall_setup(int prec, int eq, void* blk, const Dims& d, const LaunchConsts& c, cudaStream_t st);
// One step with the walls: the columns' rho_w from src, the periodic step, then the wall layers.
cudaError_t launch_wall_step(int prec, int eq, int variant, const void* src, void* dst, const Dims& d,
                             const LaunchConsts& c, double twobeta, void* blk, int* err, cudaStream_t st);

// Isothermal nonideal fluid (lb_nonideal.cu): doubles of the work buffer for this grid, and
// one step (density, fields, force, forced step).  kind: 1 van der Waals, 2 Peng-Robinson type,
// 3 Carnahan-Starling; eos = {a, b, kappa, eta}.
size_t nonideal_doubles(const Dims& d, int prec);
cudaError_t launch_nonideal_step(int prec, const void* src, void* dst, const Dims& d, const LaunchConsts& c,
                                 double twobeta, int kind, const double eos[4], double* work, int* err,
                                 cudaStream_t st);

inline dim3 step_grid(const Dims& d, int threads) {
    return dim3((unsigned)d.rows, (unsigned)((d.nx + threads - 1) / threads), 1);
}
inline int step_threads(const Dims& d) {
    return d.nx >= 128 ? 128 : ((d.nx + 31) / 32) * 32;
}

}  // namespace gblb
