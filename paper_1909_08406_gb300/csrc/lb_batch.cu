// Batched sweep: many independent RD3Q41 simulations of uneven grid sizes
// and relaxation times advanced together.
//
// Work list: every simulation's nodes are cut into tiles of TX consecutive x
// by RY consecutive rows, or (RY = 0, linear tiles) into runs of TX
// consecutive entries of its x-fastest node order that cross row ends, so a
// warp reads 32 consecutive values of each population whatever nx is; the
// tiles of all simulations are numbered back to back (tile0[k] is the first
// tile of simulation k) and a CTA finds its simulation by binary search.
// With FP32 arithmetic a thread may update one node or two (y, y + 1) with
// packed FP32x2 arithmetic.  Modes:
//   LB_BATCH_GRAPH       one batched launch per time step, the n launches
//                        captured once into a CUDA graph and replayed;
//   LB_BATCH_PERSISTENT  one cooperative launch for all n steps: CTAs stride
//                        over the work list and meet at a grid barrier between
//                        steps (bounded spin; expiry -> LB_ERR_TIMEOUT);
//   LB_BATCH_SEQUENTIAL  per simulation, one lb_step-style launch per step
//                        (the baseline).
// The tile shape (TX, RY) and the rows per thread are chosen by lb_batch_tune,
// which times each candidate on the batch itself.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gblb.h"
#include "lb_ctx.h"
#include "lb_kernels.cuh"

namespace gblb {

// Division of n < 2^31 by a run-time constant d >= 1 as one multiply and shift
// (Granlund and Montgomery, division by invariant integers using
// multiplication, 1994): with 2^k >= d and m = ceil(2^(31+k) / d),
// floor(n / d) = (n m) >> (31 + k).  Proof: write n = q d + r and
// m d = 2^(31+k) + e with 0 <= e < d <= 2^k; then
// n m / 2^(31+k) = q + (r + n e / 2^(31+k)) / d, and n e / 2^(31+k) < 1,
// so the bracket stays below d.  m < 2^32 because d > 2^(k-1) for the
// smallest such k.
struct FastDiv {
    uint32_t m, sh;
};

static FastDiv make_fastdiv(uint32_t d) {
    uint32_t k = 0;
    while ((1ull << k) < d) ++k;
    FastDiv f;
    f.m = (uint32_t)(((1ull << (31 + k)) + d - 1) / d);
    f.sh = 31 + k;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f) { return (uint32_t)(((uint64_t)n * f.m) >> f.sh); }

struct BatchSim {
    void* buf[2];
    Dims d;
    float tbf;
    double tbd;
    int64_t tile0;   // first tile of this simulation in the work list
    uint32_t units;  // entries: nodes (one row per thread) or node pairs (two rows per thread)
    uint32_t nrows;  // rows (one row per thread) or row pairs (two)
    int tiles_x;     // x-chunks per row group
    FastDiv fx, fy, fz, ft;  // division by nx, by ny (or ny / 2), by nz, by tiles_x
};

__device__ __forceinline__ int find_sim(const BatchSim* __restrict__ sims, int nsims, int64_t t) {
    int lo = 0, hi = nsims - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sims[mid].tile0 <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Node (s, z, y, x) of this thread's entry of tile t of simulation S (with two rows per thread,
// y is the first row of the pair); false past the simulation's end.  Tiles: tx x-nodes by ry
// rows (tx = 2^txs), or ry = 0: tx consecutive entries of the x-fastest order.  Every index
// is below 2^31 (lb_batch_init rejects larger simulations).
template <bool TWO>
__device__ __forceinline__ bool tile_node(const BatchSim& S, int64_t t, int tx, int txs, int ry, int& s, int& z,
                                          int& y, int& x) {
    const uint32_t local = (uint32_t)(t - S.tile0);
    uint32_t row;
    if (ry == 0) {
        const uint32_t i = local * (uint32_t)tx + threadIdx.x;
        if (i >= S.units) return false;
        row = fdiv(i, S.fx);
        x = (int)(i - row * (uint32_t)S.d.nx);
    } else {
        const uint32_t rg = fdiv(local, S.ft);
        x = (int)((local - rg * (uint32_t)S.tiles_x) * (uint32_t)tx + (threadIdx.x & (uint32_t)(tx - 1)));
        row = rg * (uint32_t)ry + (threadIdx.x >> txs);
        if (x >= S.d.nx || row >= S.nrows) return false;
    }
    const uint32_t zr = fdiv(row, S.fy);
    const uint32_t nyr = TWO ? (uint32_t)S.d.ny >> 1 : (uint32_t)S.d.ny;
    y = (int)(row - zr * nyr) * (TWO ? 2 : 1);
    const uint32_t sz = fdiv(zr, S.fz);
    z = (int)(zr - sz * (uint32_t)S.d.nz);
    s = (int)sz;
    return true;
}

template <class R>
__device__ __forceinline__ R tb_of(const BatchSim& s);
template <>
__device__ __forceinline__ float tb_of<float>(const BatchSim& s) {
    return s.tbf;
}
template <>
__device__ __forceinline__ double tb_of<double>(const BatchSim& s) {
    return s.tbd;
}

// One tile of the work list.  Ld selects the load path: the read-only path for
// one-step launches, L2-coherent loads inside the persistent kernel (a CTA may
// read, in step k + 1, lines another CTA wrote in step k).
template <class Codec, bool PROJECT, class Ld>
__device__ __forceinline__ void batch_tile(const BatchSim* __restrict__ sims, int nsims, int64_t t, int parity,
                                           const Consts<typename Codec::R>& K, int tx, int txs, int ry, int* err) {
    using R = typename Codec::R;
    using T = typename Codec::raw_t;
    const BatchSim& S = sims[find_sim(sims, nsims, t)];
    int s, z, y, x;
    if (!tile_node<false>(S, t, tx, txs, ry, s, z, y, x)) return;
    step_node<Codec, PROJECT, Ld>(static_cast<const T*>(S.buf[parity]), static_cast<T*>(S.buf[parity ^ 1]), S.d, K,
                                  tb_of<R>(S), err, s, z, y, x);
}

// Two-row tiles (FP32 arithmetic, every simulation with ny even): a tile is TX x-nodes by RY
// row pairs (or TX consecutive (row pair, x) entries); each thread updates (y, x) and
// (y + 1, x) with packed FP32x2 arithmetic.
template <class Codec, bool PROJECT, class Ld>
__device__ __forceinline__ void batch_tile2(const BatchSim* __restrict__ sims, int nsims, int64_t t, int parity,
                                            const Consts<float>& K, int tx, int txs, int ry, int* err) {
    using T = typename Codec::raw_t;
    const BatchSim& S = sims[find_sim(sims, nsims, t)];
    int s, z, y, x;
    if (!tile_node<true>(S, t, tx, txs, ry, s, z, y, x)) return;
    step_node2<Codec, PROJECT, Ld>(static_cast<const T*>(S.buf[parity]), static_cast<T*>(S.buf[parity ^ 1]), S.d, K,
                                   S.tbf, err, s, z, y, x);
}

// Resident CTAs per SM the register allocation is sized for.  One node per thread in FP32
// arithmetic fits 80 registers without spills (6 CTAs of 128 threads, 24 warps per SM); the
// persistent kernel's loop state needs 96 (5 CTAs); two nodes per thread (packed FP32x2) and
// FP64 arithmetic need about 168 (3 CTAs).
template <class Codec, bool TWO>
constexpr int batch_min_blocks(bool persistent) {
    return (TWO || sizeof(typename Codec::R) == 8) ? 3 : (persistent ? 6 : 6);
}

template <class Codec, bool PROJECT, bool TWO>
__global__ void __launch_bounds__(128, batch_min_blocks<Codec, TWO>(false)) k_batch_step(const BatchSim* __restrict__ sims, int nsims, int parity,
                                                    Consts<typename Codec::KS> K, int tx, int txs, int ry, int* err) {
    if constexpr (TWO)
        batch_tile2<Codec, PROJECT, LoadNC>(sims, nsims, blockIdx.x, parity, K, tx, txs, ry, err);
    else
        batch_tile<Codec, PROJECT, LoadNC>(sims, nsims, blockIdx.x, parity, K, tx, txs, ry, err);
}

struct GridBar {
    unsigned count;
    unsigned gen;
};

// Grid-wide barrier for a cooperative launch.  Thread 0 of each CTA arrives
// on a counter; the last arrival resets it and advances the generation; the
// others spin on the generation with a cycle budget.  Returns false (for the
// whole CTA) if the budget ran out.
__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned expected, long long limit) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &bar->gen;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

template <class Codec, bool PROJECT, bool TWO>
__global__ void __launch_bounds__(128, batch_min_blocks<Codec, TWO>(true))
    k_batch_persistent(const BatchSim* __restrict__ sims, int nsims, int64_t ntiles, int64_t nsteps, int parity0,
                       Consts<typename Codec::KS> K, int tx, int txs, int ry, int* err, GridBar* bar,
                       unsigned expected, long long limit) {
    const int nt = (int)ntiles;  // < 2^31 (the work list is checked when it is laid out)
    for (int64_t step = 0; step < nsteps; ++step) {
        const int parity = (int)((parity0 + step) & 1);
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            if constexpr (TWO)
                batch_tile2<Codec, PROJECT, LoadCG>(sims, nsims, t, parity, K, tx, txs, ry, err);
            else
                batch_tile<Codec, PROJECT, LoadCG>(sims, nsims, t, parity, K, tx, txs, ry, err);
        }
        if (step + 1 < nsteps && !grid_sync(bar, expected, limit)) {
            if (threadIdx.x == 0) atomicOr(err, 2);
            return;
        }
    }
}

template <class F>
static cudaError_t dispatch_codec(int prec, F&& f) {
    switch (prec) {
        case kF64: return f(CodecF64{});
        case kF32: return f(CodecF32{});
        case kF16: return f(CodecF16{});
        case kBF16: return f(CodecBF16{});
        default: return cudaErrorInvalidValue;
    }
}

template <class Codec>
static const Consts<typename Codec::KS>& consts_of(const LaunchConsts& c) {
    if constexpr (std::is_same<typename Codec::KS, double>::value)
        return c.kd;
    else
        return c.kf;
}

}  // namespace gblb

using namespace gblb;

// (TX, RY); RY = 0: linear tiles of TX entries
static const int kTileShapes[][2] = {{16, 4}, {16, 8}, {32, 2}, {32, 4}, {64, 1}, {64, 2}, {128, 1}, {64, 0}, {128, 0}};

static int tile_threads(int tx, int ry) { return ry == 0 ? tx : tx * ry; }

static int log2i(int v) {  // tile widths are powers of two
    int k = 0;
    while ((1 << k) < v) ++k;
    return k;
}

struct lb_batch {
    int n = 0;
    std::vector<lb_ctx*> ctx;
    int prec = 0;
    bool project = true;
    int device = 0;
    int sms = 0;
    cudaStream_t user = nullptr;
    cudaStream_t ps = nullptr;  // private stream (graph capture needs a non-legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
    // One work list per launch mode: the graph-replayed batched launch and the persistent
    // kernel are tuned separately (they differ in registers, occupancy and load path).
    struct Plan {
        int tx = 32, ry = 4;
        bool two_rows = false;  // two rows per thread (FP32x2)
        int64_t ntiles = 0;
        BatchSim* d_sims = nullptr;
    };
    Plan gp, pp;  // LB_BATCH_GRAPH, LB_BATCH_PERSISTENT
    std::vector<BatchSim> h_sims;
    bool two_rows_ok = false;  // FP32 arithmetic and every simulation with ny even
    int* d_err = nullptr;
    GridBar* d_bar = nullptr;
    long long wait_limit = 4000000000LL;
    unsigned extra_arrivals = 0;
    struct GraphEntry {  // captured for the graph plan in use; dropped when it changes
        int64_t steps;
        int parity;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    int persistent_graph = -1;  // -1 untried, 0 direct launch, 1 captured in a graph
    std::string msg;
};

static std::string g_batch_init_msg;

static lb_status bfail(lb_batch* b, lb_status s, const std::string& m) {
    if (b)
        b->msg = m;
    else
        g_batch_init_msg = m;
    return s;
}

#define BCK(b, call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,               \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

// Lay out the work list of plan P for tile shape (tx, ry) and rows per thread, and upload it.
static lb_status plan(lb_batch* b, lb_batch::Plan& P, int tx, int ry, bool two_rows) {
    int64_t t = 0;
    for (int k = 0; k < b->n; ++k) {
        BatchSim& s = b->h_sims[k];
        const lb_ctx* c = b->ctx[k];
        s.buf[0] = c->buf[0];
        s.buf[1] = c->buf[1];
        s.d = c->d;
        s.tbd = c->twobeta;
        s.tbf = (float)c->twobeta;
        s.tiles_x = (int)((c->d.nx + tx - 1) / tx);
        s.tile0 = t;
        const int64_t rows = two_rows ? c->d.rows / 2 : c->d.rows;
        s.units = (uint32_t)(rows * c->d.nx);  // < 2^31 (lb_batch_init)
        s.nrows = (uint32_t)rows;
        s.fx = make_fastdiv((uint32_t)c->d.nx);
        s.fy = make_fastdiv((uint32_t)(two_rows ? c->d.ny / 2 : c->d.ny));
        s.fz = make_fastdiv((uint32_t)c->d.nz);
        s.ft = make_fastdiv((uint32_t)s.tiles_x);
        t += ry == 0 ? ((int64_t)s.units + tx - 1) / tx : (int64_t)s.tiles_x * ((rows + ry - 1) / ry);
    }
    if (t > 0x7fffffffLL) return bfail(b, LB_ERR_ARG, "batch work list too long for one launch");
    P.ntiles = t;
    P.tx = tx;
    P.ry = ry;
    P.two_rows = two_rows;
    BCK(b, cudaMemcpyAsync(P.d_sims, b->h_sims.data(), sizeof(BatchSim) * b->n, cudaMemcpyHostToDevice, b->ps));
    BCK(b, cudaStreamSynchronize(b->ps));
    if (&P == &b->gp) {
        for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
        b->graphs.clear();
    }
    return LB_OK;
}

static cudaError_t launch_batch_step(lb_batch* b, int parity, cudaStream_t st) {
    const LaunchConsts& lc = lattice_consts();
    return dispatch_codec(b->prec, [&](auto codec) {
        using C = decltype(codec);
        const lb_batch::Plan& P = b->gp;
        const unsigned grid = (unsigned)P.ntiles, block = (unsigned)tile_threads(P.tx, P.ry);
        if constexpr (std::is_same<typename C::R, float>::value) {
            if (P.two_rows) {
                if (b->project)
                    k_batch_step<C, true, true><<<grid, block, 0, st>>>(P.d_sims, b->n, parity, consts_of<C>(lc),
                                                                        P.tx, log2i(P.tx), P.ry, b->d_err);
                else
                    k_batch_step<C, false, true><<<grid, block, 0, st>>>(P.d_sims, b->n, parity, consts_of<C>(lc),
                                                                         P.tx, log2i(P.tx), P.ry, b->d_err);
                return cudaGetLastError();
            }
        }
        if (b->project)
            k_batch_step<C, true, false><<<grid, block, 0, st>>>(P.d_sims, b->n, parity, consts_of<C>(lc), P.tx,
                                                                 log2i(P.tx), P.ry, b->d_err);
        else
            k_batch_step<C, false, false><<<grid, block, 0, st>>>(P.d_sims, b->n, parity, consts_of<C>(lc), P.tx,
                                                                  log2i(P.tx), P.ry, b->d_err);
        return cudaGetLastError();
    });
}

static cudaError_t launch_persistent(lb_batch* b, int64_t nsteps, int parity, cudaStream_t st, int* grid_out) {
    const LaunchConsts& lc = lattice_consts();
    return dispatch_codec(b->prec, [&](auto codec) -> cudaError_t {
        using C = decltype(codec);
        void (*kern)(const BatchSim*, int, int64_t, int64_t, int, Consts<typename C::KS>, int, int, int, int*,
                     GridBar*, unsigned, long long) =
            b->project ? k_batch_persistent<C, true, false> : k_batch_persistent<C, false, false>;
        if constexpr (std::is_same<typename C::R, float>::value) {
            if (b->pp.two_rows)
                kern = b->project ? k_batch_persistent<C, true, true> : k_batch_persistent<C, false, true>;
        }
        int per_sm = 0;
        const lb_batch::Plan& P = b->pp;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tile_threads(P.tx, P.ry), 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        int64_t grid = (int64_t)per_sm * b->sms;
        if (grid > P.ntiles) grid = P.ntiles;
        *grid_out = (int)grid;
        unsigned expected = (unsigned)grid + b->extra_arrivals;
        e = cudaMemsetAsync(b->d_bar, 0, sizeof(GridBar), st);
        if (e != cudaSuccess) return e;
        const BatchSim* sims = P.d_sims;
        int nsims = b->n;
        int64_t ntiles = P.ntiles;
        Consts<typename C::KS> K = consts_of<C>(lc);
        int tx = P.tx, txs = log2i(P.tx), ry = P.ry;
        int* err = b->d_err;
        GridBar* bar = b->d_bar;
        long long limit = b->wait_limit;
        void* args[] = {(void*)&sims, (void*)&nsims, (void*)&ntiles, (void*)&nsteps, (void*)&parity, (void*)&K,
                        (void*)&tx, (void*)&txs, (void*)&ry, (void*)&err, (void*)&bar, (void*)&expected,
                        (void*)&limit};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)tile_threads(tx, ry));
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelExC(&cfg, (const void*)kern, args);
    });
}

extern "C" {

lb_status lb_batch_init(lb_batch** out, int nsims, const lb_grid* grids, const double* tau, lb_precision precision,
                        unsigned flags, void* cuda_stream) {
    if (!out || nsims < 1 || !grids || !tau) return bfail(nullptr, LB_ERR_ARG, "lb_batch_init: bad argument");
    *out = nullptr;
    if (flags & (LB_FLAG_ENTROPIC | LB_FLAG_ENTROPIC_PATH))
        return bfail(nullptr, LB_ERR_ARG, "lb_batch_init: the exact entropic equilibrium is a single-grid mode");
    for (int k = 0; k < nsims; ++k) {
        const lb_grid& g = grids[k];
        if (g.nx >= 1 && g.ny >= 1 && g.nz >= 1 && g.nx < (1 << 30) && g.ny < (1 << 30) && g.nz < (1 << 30) &&
            2.0 * (double)g.nx * (double)g.ny * (double)g.nz >= 2147483648.0)
            return bfail(nullptr, LB_ERR_ARG,
                         "lb_batch_init: simulation " + std::to_string(k) + " has 2^31 nodes or more (single-grid only)");
    }
    lb_batch* b = new lb_batch();
    b->n = nsims;
    b->prec = (int)precision;
    b->project = !(flags & LB_FLAG_PAPER_LITERAL);
    b->user = (cudaStream_t)cuda_stream;
    for (int k = 0; k < nsims; ++k) {
        lb_ctx* c = nullptr;
        lb_status s = lb_init(&c, grids[k], LB_RD3Q41, 0.0, tau[k], precision, flags, cuda_stream);
        if (s != LB_OK) {
            std::string m = std::string("lb_batch_init: simulation ") + std::to_string(k) + ": " + lb_last_error(nullptr);
            for (auto* p : b->ctx) lb_destroy(p);
            delete b;
            return bfail(nullptr, s, m);
        }
        b->ctx.push_back(c);
    }
    b->h_sims.resize(nsims);
    b->two_rows_ok = precision != LB_F64;
    for (auto* c : b->ctx) b->two_rows_ok = b->two_rows_ok && c->d.ny % 2 == 0 && c->d.plane < ((int64_t)1 << 32);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->ps, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
    if (e == cudaSuccess) e = cudaMalloc(&b->gp.d_sims, sizeof(BatchSim) * nsims);
    if (e == cudaSuccess) e = cudaMalloc(&b->pp.d_sims, sizeof(BatchSim) * nsims);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, sizeof(GridBar));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        lb_batch_destroy(b);
        return bfail(nullptr, LB_ERR_CUDA, std::string("lb_batch_init: ") + cudaGetErrorString(e));
    }
    lb_status s = plan(b, b->gp, 32, 4, b->two_rows_ok);
    if (s == LB_OK) s = plan(b, b->pp, 32, 4, b->two_rows_ok);
    if (s != LB_OK) {
        std::string m = b->msg;
        lb_batch_destroy(b);
        return bfail(nullptr, s, m);
    }
    *out = b;
    return LB_OK;
}

int lb_batch_size(const lb_batch* b) { return b ? b->n : -1; }

lb_ctx* lb_batch_sim(lb_batch* b, int sim) { return (b && sim >= 0 && sim < b->n) ? b->ctx[sim] : nullptr; }

lb_status lb_batch_set_tile(lb_batch* b, int tx, int ry) {
    if (!b) return LB_ERR_ARG;
    bool known = false;
    for (auto& t : kTileShapes) known |= (t[0] == tx && t[1] == ry);
    if (!known) return bfail(b, LB_ERR_ARG, "lb_batch_set_tile: not one of the tile shapes");
    BCK(b, cudaSetDevice(b->device));
    lb_status s = plan(b, b->gp, tx, ry, b->gp.two_rows);
    return s != LB_OK ? s : plan(b, b->pp, tx, ry, b->pp.two_rows);
}

lb_status lb_batch_get_tile(const lb_batch* b, int* tx, int* ry) {
    if (!b) return LB_ERR_ARG;
    if (tx) *tx = b->gp.tx;
    if (ry) *ry = b->gp.ry;
    return LB_OK;
}

lb_status lb_batch_set_rows(lb_batch* b, int rows_per_thread) {
    if (!b || (rows_per_thread != 1 && rows_per_thread != 2)) return bfail(b, LB_ERR_ARG, "lb_batch_set_rows: 1 or 2");
    if (rows_per_thread == 2 && !b->two_rows_ok)
        return bfail(b, LB_ERR_ARG, "lb_batch_set_rows: two rows per thread need FP32 arithmetic and ny even");
    BCK(b, cudaSetDevice(b->device));
    lb_status s = plan(b, b->gp, b->gp.tx, b->gp.ry, rows_per_thread == 2);
    return s != LB_OK ? s : plan(b, b->pp, b->pp.tx, b->pp.ry, rows_per_thread == 2);
}

int lb_batch_get_rows(const lb_batch* b) { return b ? (b->gp.two_rows ? 2 : 1) : -1; }

lb_status lb_batch_get_plan(const lb_batch* b, int mode, int* tx, int* ry, int* rows_per_thread) {
    if (!b || (mode != LB_BATCH_GRAPH && mode != LB_BATCH_PERSISTENT)) return LB_ERR_ARG;
    const lb_batch::Plan& P = mode == LB_BATCH_GRAPH ? b->gp : b->pp;
    if (tx) *tx = P.tx;
    if (ry) *ry = P.ry;
    if (rows_per_thread) *rows_per_thread = P.two_rows ? 2 : 1;
    return LB_OK;
}

// Time `reps` launches of one batched step in the given mode with the current plans (after one
// untimed launch); the trial steps read buf[cur] and write buf[1 - cur] without flipping.
static lb_status time_trial(lb_batch* b, int mode, int parity, int reps, float* ms) {
    int grid = 0;
    auto launch = [&]() {
        return mode == LB_BATCH_GRAPH ? launch_batch_step(b, parity, b->ps) : launch_persistent(b, 1, parity, b->ps, &grid);
    };
    BCK(b, launch());
    BCK(b, cudaEventRecord(b->t0, b->ps));
    for (int r = 0; r < reps; ++r) BCK(b, launch());
    BCK(b, cudaEventRecord(b->t1, b->ps));
    BCK(b, cudaEventSynchronize(b->t1));
    BCK(b, cudaEventElapsedTime(ms, b->t0, b->t1));
    *ms /= reps;
    return LB_OK;
}

lb_status lb_batch_tune(lb_batch* b, int reps, int* tx_out, int* ry_out, double* ms_out) {
    if (!b) return LB_ERR_ARG;
    BCK(b, cudaSetDevice(b->device));
    if (reps < 1) reps = 3;
    // the trial steps leave the state unchanged (see time_trial)
    BCK(b, cudaEventRecord(b->ev_in, b->user));
    BCK(b, cudaStreamWaitEvent(b->ps, b->ev_in, 0));
    const int parity = b->ctx[0]->cur;
    float best_ms = 0.f;
    for (int mode : {LB_BATCH_GRAPH, LB_BATCH_PERSISTENT}) {
        lb_batch::Plan& P = mode == LB_BATCH_GRAPH ? b->gp : b->pp;
        float best = 1e30f;
        int bt = P.tx, br = P.ry;
        bool b2 = P.two_rows;
        for (int two = 0; two <= (b->two_rows_ok ? 1 : 0); ++two) {
            for (auto& shape : kTileShapes) {
                lb_status s = plan(b, P, shape[0], shape[1], two != 0);
                if (s != LB_OK) return s;
                float ms = 0.f;
                s = time_trial(b, mode, parity, reps, &ms);
                if (s != LB_OK) return s;
                if (ms < best) {
                    best = ms;
                    bt = shape[0];
                    br = shape[1];
                    b2 = two != 0;
                }
            }
        }
        lb_status s = plan(b, P, bt, br, b2);
        if (s != LB_OK) return s;
        if (mode == LB_BATCH_GRAPH) best_ms = best;
    }
    if (tx_out) *tx_out = b->gp.tx;
    if (ry_out) *ry_out = b->gp.ry;
    if (ms_out) *ms_out = best_ms;
    return LB_OK;
}

lb_status lb_batch_set_wait(lb_batch* b, long long limit_cycles, unsigned extra_arrivals) {
    if (!b || limit_cycles < 1) return LB_ERR_ARG;
    b->wait_limit = limit_cycles;
    b->extra_arrivals = extra_arrivals;
    return LB_OK;
}

lb_status lb_batch_step(lb_batch* b, int64_t nsteps, int mode) {
    if (!b || nsteps < 0) return bfail(b, LB_ERR_ARG, "lb_batch_step: bad argument");
    if (nsteps == 0) return LB_OK;
    for (auto* c : b->ctx)
        if (c->walls || c->nonideal || c->sr)
            return bfail(b, LB_ERR_STATE,
                         "lb_batch_step: a simulation of the batch has walls, the nonideal mode or stochastic rounding");
    BCK(b, cudaSetDevice(b->device));
    const int parity = b->ctx[0]->cur;
    if (mode == LB_BATCH_SEQUENTIAL) {
        for (auto* c : b->ctx) {
            lb_status s = lb_step(c, nsteps);
            if (s != LB_OK) return bfail(b, s, lb_last_error(c));
        }
        return LB_OK;
    }
    BCK(b, cudaEventRecord(b->ev_in, b->user));
    BCK(b, cudaStreamWaitEvent(b->ps, b->ev_in, 0));
    if (mode == LB_BATCH_GRAPH) {
        cudaGraphExec_t exec = nullptr;
        for (auto& g : b->graphs)
            if (g.steps == nsteps && g.parity == parity) exec = g.exec;
        if (!exec) {
            cudaGraph_t graph = nullptr;
            BCK(b, cudaStreamBeginCapture(b->ps, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int64_t t = 0; t < nsteps && e == cudaSuccess; ++t) e = launch_batch_step(b, parity ^ (int)(t & 1), b->ps);
            cudaError_t e2 = cudaStreamEndCapture(b->ps, &graph);
            if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("batched launch during capture: ") + cudaGetErrorString(e));
            if (e2 != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e2));
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
            if (b->graphs.size() >= 8) {
                cudaGraphExecDestroy(b->graphs.front().exec);
                b->graphs.erase(b->graphs.begin());
            }
            b->graphs.push_back({nsteps, parity, exec});
        }
        BCK(b, cudaGraphLaunch(exec, b->ps));
    } else if (mode == LB_BATCH_PERSISTENT) {
        int grid = 0;
        BCK(b, launch_persistent(b, nsteps, parity, b->ps, &grid));
    } else {
        return bfail(b, LB_ERR_ARG, "lb_batch_step: unknown mode");
    }
    BCK(b, cudaEventRecord(b->ev_out, b->ps));
    BCK(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
    for (auto* c : b->ctx) {
        c->cur ^= (int)(nsteps & 1);
        c->time += nsteps;
    }
    return LB_OK;
}

lb_status lb_batch_sync(lb_batch* b) {
    if (!b) return LB_ERR_ARG;
    BCK(b, cudaSetDevice(b->device));
    BCK(b, cudaStreamSynchronize(b->ps));
    BCK(b, cudaStreamSynchronize(b->user));
    int h = 0;
    BCK(b, cudaMemcpy(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & 2) return bfail(b, LB_ERR_TIMEOUT, "a grid barrier of the persistent batch kernel gave up waiting");
    if (h) return bfail(b, LB_ERR_UNSTABLE, "a node reached rho <= 0, theta <= 0 or a non-finite moment");
    for (auto* c : b->ctx) {
        lb_status s = lb_sync(c);
        if (s != LB_OK) return bfail(b, s, lb_last_error(c));
    }
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch* b) {
    if (!b) return LB_OK;
    cudaSetDevice(b->device);
    if (b->ps) cudaStreamSynchronize(b->ps);
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
    for (auto* c : b->ctx) lb_destroy(c);
    if (b->ps) cudaStreamDestroy(b->ps);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    cudaFree(b->gp.d_sims);
    cudaFree(b->pp.d_sims);
    cudaFree(b->d_err);
    cudaFree(b->d_bar);
    delete b;
    return LB_OK;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->msg.c_str() : g_batch_init_msg.c_str(); }

}  // extern "C"
