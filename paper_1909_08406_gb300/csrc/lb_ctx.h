// Internal definition of the solver context (opaque in gblb.h), shared by the
// single-grid API and the batched API.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "gblb.h"
#include "lb_launch.h"

struct lb_ctx {
    lb_grid g;
    gblb::Dims d;
    int prec;
    int eq;  // equilibrium kind: 0 as printed, 1 with the momentum projection, 2 exact entropic
    int variant;
    double tau, twobeta;
    cudaStream_t stream;
    int device;
    void* buf[2];  // ping-pong population buffers; buf[cur] holds the current state
    int cur;
    size_t esize;
    int* d_err;    // sticky device error word: bit 0 unstable node, bit 1 wait timeout
    double* d_partials;
    int nblocks;
    double* d_out5;
    double* d_stage;
    int64_t stage_doubles;
    int64_t time;
    int walls = 0;           // kinetic walls normal to z (lb_set_walls) instead of the periodic wrap
    void* d_wall = nullptr;  // the walls' device block (lb_walls.cu)
    int nonideal = 0;          // isothermal nonideal fluid: 0 off, else its equation of state (lb_set_nonideal)
    double ni_eos[4] = {0, 0, 0, 0};  // a, b, kappa, eta
    double* d_ni = nullptr;    // its work buffer (lb_nonideal.cu)
    int sr = 0;                // stochastic rounding of the BF16 store (lb_set_stochastic_rounding)
    uint64_t sr_seed = 0;
    uint32_t sr_t = 0;         // steps taken since it was enabled
    std::string msg;
};

namespace gblb {
const LaunchConsts& lattice_consts();
}
