"""Error of the reduced-precision storage modes over many steps, against the GPU
FP64 mode (itself matched to the FP64 oracle to 1e-12), on the thermoacoustic
case (density pulse 1e-2, sigma 8 cells, plus a 1e-3 temperature field).

Bound, from the arithmetic.  Each step rounds every stored deviation
h_i = f_i / w_i - 1 once, to nearest: an error of zero mean and variance at most
(u h_i)^2 / 3, u the storage format's unit roundoff (2^-11 FP16, 2^-8 BF16).
The linearised update is a contraction in the w-weighted norm
||h||_w^2 = sum_nodes sum_i w_i h_i^2 (streaming permutes, BGK at 0 <= 2 beta <= 2
shrinks the non-equilibrium part, the equilibrium being the w-orthogonal
projection onto 1, c, c^2 / theta0 - 3), and per node |sum_i w_i dh_i| <= the
node's w-norm of dh (Cauchy-Schwarz, sum w_i = 1).  With errors uncorrelated
from step to step the density error after t steps is then, in expectation,
    ||d rho_t||_2 <= sqrt(t / 3) u ||h_0||_w,
and for the initial equilibrium ||h_0||_w^2 = sum (drho^2 + |u|^2 / theta0
+ 3/2 (dtheta / theta0)^2) to leading order.  The test allows twice that
(non-linear terms, FP32 arithmetic).  The bound ignores the damping of the
short-wave rounding noise, so the measured errors sit far below it (about 1/60
at 128^3 and 200 steps); the tight check is the next one: because the error is
storage rounding, the BF16 and FP16 errors must stand near the ratio of their
unit roundoffs, 8 (measured 10.4 for the density, 10.9 for the temperature).

Stochastic rounding of the BF16 store (lb_set_stochastic_rounding) has zero mean
by construction and variance p(1 - p) s^2 <= s^2 / 4 per value, s = 2 u |h| the
BF16 spacing, so the same argument gives ||d rho_t||_2 <= sqrt(t) u ||h_0||_w
(again allowed twice).  Round to nearest repeats its error at a node whose h
changes by less than a spacing from one step to the next, and that part grows
like t, not sqrt(t): over 1000 steps at 128^3 the stochastic store must be at
least twice as accurate (measured 2.8x for the density, 2.9x for the
temperature; 1.7x at 256^3 and 500 steps)."""
import math

import pytest

from paper_1909_08406_gb300 import accuracy_report
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

N, STEPS = 128, 200
LONG_STEPS = 1000
UNIT_ROUNDOFF = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "bf16sr": 2.0 ** -8}
# expected squared error per rounding, in units of (u h)^2: 1/3 to nearest, at most 1 stochastically
VARIANCE = {"f16": 1.0 / 3.0, "bf16": 1.0 / 3.0, "bf16sr": 1.0}


def _h0_w(fields, th0):
    return math.sqrt(float(((fields["rho"] - 1.0) ** 2).sum()
                           + (fields["u"] ** 2).sum() / th0
                           + 1.5 * ((fields["theta"] / th0 - 1.0) ** 2).sum()))


@pytest.fixture(scope="module")
def errors():
    th0 = lb.lb_theta0()
    fields = wl.thermoacoustic_pulse(N, th0, device="cuda")
    h0 = _h0_w(fields, th0)
    out = accuracy_report.compare(N, STEPS, ("f32", "f16", "bf16", "bf16sr"), fields)
    print({"h0_w": h0, **out})
    return out, h0, out["f64"]["l2_rho_fluct"]


@pytest.fixture(scope="module")
def long_errors():
    th0 = lb.lb_theta0()
    fields = wl.thermoacoustic_pulse(N, th0, device="cuda")
    h0 = _h0_w(fields, th0)
    out = accuracy_report.compare(N, LONG_STEPS, ("bf16", "bf16sr"), fields)
    print({"h0_w": h0, **out})
    return out, h0, out["f64"]["l2_rho_fluct"]


@pytest.mark.parametrize("prec", ["f16", "bf16", "bf16sr"])
def test_density_error_within_rounding_bound(prec, errors):
    out, h0, nr = errors
    err = out[prec]["rel_l2_rho_fluct"] * nr
    bound = 2.0 * math.sqrt(STEPS * VARIANCE[prec]) * UNIT_ROUNDOFF[prec] * h0
    assert err <= bound, (prec, err, bound, out[prec])


def test_stochastic_rounding_error_grows_like_a_random_walk(long_errors):
    out, h0, nr = long_errors
    err = out["bf16sr"]["rel_l2_rho_fluct"] * nr
    assert err <= 2.0 * math.sqrt(LONG_STEPS) * UNIT_ROUNDOFF["bf16sr"] * h0, out["bf16sr"]
    for key in ("rel_l2_rho_fluct", "rel_l2_theta_fluct"):
        assert out["bf16"][key] >= 2.0 * out["bf16sr"][key], (key, out)


def test_fp32_density_error_meets_target(errors):
    """FP32 storage: the error is the FP32 evaluation of the update, whose rounding is
    relative to O(1) quantities (moments, weights), not to h, so the storage model above does
    not bound it; the stated target is 1e-4 of the density fluctuation (measured: ~6e-6)."""
    out, _, _ = errors
    assert out["f32"]["rel_l2_rho_fluct"] <= 1e-4, out["f32"]
    assert out["f32"]["rel_l2_theta_fluct"] <= 1e-4, out["f32"]


def test_16bit_errors_scale_with_unit_roundoff(errors):
    out, _, _ = errors
    ratio = out["bf16"]["rel_l2_rho_fluct"] / out["f16"]["rel_l2_rho_fluct"]
    assert 4.0 <= ratio <= 16.0, (ratio, out)
    ratio_t = out["bf16"]["rel_l2_theta_fluct"] / out["f16"]["rel_l2_theta_fluct"]
    assert 4.0 <= ratio_t <= 16.0, (ratio_t, out)
