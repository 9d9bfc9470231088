"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/*.h (lb_* and sg_*), reports the paper's velocity set, and
rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b((?:lb|sg)_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_1909_08406_gb300 import build, lb
    build.build()
    return lb.lib()


def test_library_exports_every_declared_symbol(L):
    names = _declared_symbols()
    assert "lb_init" in names and "lb_step" in names and "sg_conv3d_fwd" in names and "sg_set_conv_impl" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_velocity_set_matches_oracle(L):
    from paper_1909_08406_gb300 import lb
    c2, w = lb.lb_velocity_set()
    c2o, wo, _ = oracle.velocities()
    by_vel = {tuple((2 * c).astype(int)): wt for c, wt in zip(c2o, wo)}
    assert {tuple(v) for v in c2} == set(by_vel)
    for v, wt in zip(c2, w):
        assert wt == pytest.approx(by_vel[tuple(v)], rel=0, abs=1e-17)
    # +-c pairs at 2k+1, 2k+2
    for k in range(20):
        assert np.array_equal(c2[2 * k + 1], -c2[2 * k + 2])
    assert lb.lb_theta0() == pytest.approx(oracle.theta0(), rel=1e-15)


def test_init_rejects_bad_arguments(L):
    from paper_1909_08406_gb300 import lb
    th = lb.lb_theta0()
    with pytest.raises(lb.LbError) as e:
        lb.lb_init((8, 8, 8), tau=0.5, theta0=th * (1 + 1e-9))
    assert e.value.status == -4
    with pytest.raises(lb.LbError) as e:
        lb.lb_init((8, 8, 8), tau=0.5, velocity_set=27)
    assert e.value.status == -1
    with pytest.raises(lb.LbError) as e:
        lb.lb_init((0, 8, 8), tau=0.5)
    assert e.value.status == -1
    with pytest.raises(lb.LbError) as e:
        lb.lb_init((8, 8, 8), tau=-1.0)
    assert e.value.status == -1
    with pytest.raises(lb.LbError) as e:
        lb.lb_init((8, 8, 8), tau=0.5, precision=7)
    assert e.value.status == -1
    assert "theta" in lb.lb_last_error() or "precision" in lb.lb_last_error()


def test_null_context_is_rejected(L):
    assert L.lb_step(None, ctypes.c_int64(1)) == -1
    assert L.lb_sync(None) == -1
    assert L.lb_destroy(None) == 0


def test_conv_impl_switch(L):
    from paper_1909_08406_gb300 import sg
    prev = sg.set_conv_impl(sg.CONV_MMA_SYNC)
    assert sg.set_conv_impl(prev) == sg.CONV_MMA_SYNC
    with pytest.raises(ValueError):
        sg.set_conv_impl(7)


def test_batch_rejects_members_of_2_31_nodes(L):
    """The batched kernels index a simulation's nodes in 32 bits: a member of 2^31 nodes or
    more is refused before anything is allocated."""
    from paper_1909_08406_gb300 import lb
    with pytest.raises(lb.LbError) as e:
        lb.lb_batch_init([(8, 8, 8), (1024, 1024, 1024)], [0.6, 0.7], "f32")
    assert e.value.status == -1
    assert "2^31" in str(e.value)
    assert L.lb_batch_get_rows(None) == -1
    assert L.lb_batch_get_plan(None, 0, None, None, None) == -1


def test_wall_and_grid_entry_points_reject_null(L):
    from paper_1909_08406_gb300 import lb
    lb.lib()
    assert L.lb_set_walls(None, 1, None, None) == -1
    assert L.lb_set_wall_columns(None, None, None) == -1
    assert L.lb_wall_density(None, None) == -1
    assert L.lb_get_grid(None, None) == -1


@pytest.mark.parametrize("eos", ["vdw", "peng_robinson", "carnahan_starling"])
@pytest.mark.parametrize("theta_star,rho_c", [(0.9, 1.0), (0.8, 0.13)])
def test_nonideal_constants_match_oracle(L, eos, theta_star, rho_c):
    """lb_nonideal_constants (host only) against the oracle's equations of state."""
    from oracle import nonideal as ni
    from paper_1909_08406_gb300 import lb
    cls = {"vdw": ni.VdW, "peng_robinson": ni.PengRobinson, "carnahan_starling": ni.CarnahanStarling}[eos]
    e = cls(theta_star, rho_c=rho_c)
    a, b = lb.lb_nonideal_constants(eos, theta_star, rho_c)
    assert a == pytest.approx(e.a, rel=1e-12) and b == pytest.approx(e.b, rel=1e-12)


def test_nonideal_constants_reject_bad_arguments(L):
    from paper_1909_08406_gb300 import lb
    for args in [(0, 0.9, 1.0), (4, 0.9, 1.0), (1, 0.0, 1.0), (1, 0.9, -1.0), (2, float("nan"), 1.0)]:
        with pytest.raises(lb.LbError) as e:
            lb.lb_nonideal_constants(*args)
        assert e.value.status == -1


@pytest.mark.parametrize("header", ["gblb.h", "gblb_surrogate.h"])
@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++11")])
def test_public_headers_compile_as_c_and_cpp(header, lang, std, tmp_path):
    """The boundary's headers are plain C: a C99 or C++11 program that includes one and calls
    nothing still compiles (no torch, CUDA or C++-only types in the signatures)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / ("main." + ("c" if lang == "c" else "cpp"))
    src.write_text('#include "%s"\nint main(void) { return 0; }\n' % header)
    subprocess.run([cc, std, "-Wall", "-Werror", "-pedantic", "-I", inc, "-fsyntax-only", str(src)], check=True,
                   capture_output=True)


C_CONSUMER = r"""
#include <math.h>
#include <stdio.h>
#include "gblb.h"
int main(void) {
    int c2[41 * 3];
    double w[41], sum = 0.0, a = 0.0, b = 0.0;
    if (lb_velocity_set(c2, w) != LB_OK) return 1;
    for (int i = 0; i < 41; ++i) sum += w[i];
    if (lb_nonideal_constants(LB_EOS_VAN_DER_WAALS, 0.9, 1.0, &a, &b) != LB_OK) return 2;
    if (lb_nonideal_constants(7, 0.9, 1.0, &a, &b) != LB_ERR_ARG) return 3;
    printf("%.17g %.17g %.17g\n", lb_theta0(), sum, b);
    return 0;
}
"""


def test_plain_c_program_links_and_calls_the_library(L, tmp_path):
    """A C99 program links against the shared library and calls its host-only entry points
    (velocity set, theta0, equation-of-state constants): the boundary needs no Python."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(L._name)
    src, exe = tmp_path / "consumer.c", tmp_path / "consumer"
    src.write_text(C_CONSUMER)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lgblb", "-Wl,-rpath," + libdir, "-lm"], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    theta0, wsum, b = (float(v) for v in out)
    assert theta0 == pytest.approx(oracle.theta0(), rel=1e-15)
    assert wsum == pytest.approx(1.0, abs=1e-15)
    assert b == pytest.approx(1.0 / 3.0, rel=1e-15)


def test_entropic_path_flag_rules_on_the_host(L):
    """LB_FLAG_ENTROPIC_PATH needs LB_FLAG_ENTROPIC, and batches refuse it, before any device work."""
    from paper_1909_08406_gb300 import lb
    with pytest.raises(lb.LbError) as e:
        lb.lb_init((8, 8, 8), tau=0.5, flags=lb.LB_FLAG_ENTROPIC_PATH)
    assert e.value.status == -1 and "LB_FLAG_ENTROPIC" in str(e.value)
    with pytest.raises(lb.LbError) as e:
        lb.lb_batch_init([(8, 8, 8)], [0.6], "f32", flags=lb.LB_FLAG_ENTROPIC | lb.LB_FLAG_ENTROPIC_PATH)
    assert e.value.status == -1


def test_relabel_and_x_period_reject_bad_arguments(L):
    """sg_relabel and the convolutions check dilations, sizes, aliasing and the x period before
    launching anything (the pointers below are never dereferenced)."""
    from paper_1909_08406_gb300 import sg
    sg._L()
    a, b = ctypes.c_void_p(4096), ctypes.c_void_p(8192)
    nat = sg.SgShape(1, 8, 16, 64, 0)
    assert L.sg_relabel(nat, 64, 1, 3, a, b, None) == -1        # dilation not a power of two
    assert L.sg_relabel(nat, 64, 1, 16, a, b, None) == -1       # dilation above 8
    assert L.sg_relabel(nat, 48, 1, 2, a, b, None) == -1        # 3 chunks per voxel
    assert L.sg_relabel(nat, 64, 1, 2, a, a, None) == -1        # in place
    assert L.sg_relabel(nat, 64, 1, 2, ctypes.c_void_p(4100), b, None) == -1  # unaligned
    assert L.sg_relabel(sg.SgShape(1, 6, 16, 64, 0), 64, 1, 4, a, b, None) == -1  # nz % d
    assert L.sg_relabel(sg.SgShape(1, 8, 16, 32, 0), 64, 1, 2, a, b, None) == -1  # nx != 64
    for xper in (4, 24, 128, -8):
        s = sg.SgShape(1, 8, 16, 64, xper)
        assert L.sg_conv3d_fwd(s, 32, 32, a, b, None, 0, 0, None, None, b, None) == -1, xper
        assert L.sg_conv3d_fwd_f32(s, 32, 32, a, b, None, b, None) == -1, xper
        assert L.sg_conv3d_wgrad(s, 32, 32, a, b, b, None, a, None) == -1, xper
