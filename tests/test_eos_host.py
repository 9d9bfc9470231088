"""The kernel's equations of state (``csrc/lb_eos.cuh``, the functions the nonideal
density kernel calls) compiled for the host with nvcc and compared with the
oracle's ``oracle/nonideal.py`` on a density sweep: FP64 to round-off, FP32 to
its rounding.  No GPU is used."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import nonideal as ni

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1909_08406_gb300", "csrc")

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include "lb_eos.cuh"
int main(int argc, char** argv) {
    const gblb::NiEos e{atof(argv[2]), atof(argv[3]), atof(argv[4]), 0.0, 0.5, atoi(argv[1])};
    for (int i = 5; i < argc; ++i) {
        const double r = atof(argv[i]);
        double mu, F;
        float muf, Ff;
        gblb::ni_eos<double>(r, e, mu, F);
        gblb::ni_eos<float>((float)r, e, muf, Ff);
        printf("%.17g %.17g %.9g %.9g\n", mu, F, (double)muf, (double)Ff);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def eos_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("eos")
    src, exe = d / "eos_host.cu", d / "eos_host"
    src.write_text(DRIVER)
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-gencode", "arch=compute_103a,code=sm_103a", "-o",
                    str(exe), str(src)], check=True, capture_output=True)
    return str(exe)


@pytest.mark.parametrize("kind,name,theta_star", [(1, "vdw", 0.9), (2, "peng_robinson", 0.9), (2, "peng_robinson", 0.75),
                                                  (3, "carnahan_starling", 0.9), (3, "carnahan_starling", 0.7)])
def test_kernel_equation_of_state_matches_oracle(eos_exe, kind, name, theta_star):
    cls = {"vdw": ni.VdW, "peng_robinson": ni.PengRobinson, "carnahan_starling": ni.CarnahanStarling}[name]
    e = cls(theta_star)
    rho = np.linspace(0.02, 0.9 * min(e.rho_max(), 4.5), 97)
    args = ["%.17g" % v for v in [e.a, e.b, oracle.theta0()] + list(rho)]
    out = subprocess.run([eos_exe, str(kind)] + args,
                         check=True, capture_output=True, text=True).stdout
    got = np.array([[float(v) for v in line.split()] for line in out.strip().splitlines()])
    mu, F = e.mu_nid(rho), e.F_nid(rho)
    scale = oracle.theta0() * (1 + rho)  # the magnitude of theta0 rho (ln rho - 1) the lattice carries
    assert np.abs(got[:, 0] - mu).max() <= 1e-14 * scale.max()
    assert np.abs(got[:, 1] - F).max() <= 1e-14 * (scale * rho).max()
    # FP32: the density itself is rounded to 2^-24 relative; the logarithms and divisions of
    # the singular factors amplify that by at most about 10 over this range
    assert (np.abs(got[:, 2] - mu) / scale).max() <= 2e-6
    assert (np.abs(got[:, 3] - F) / (scale * rho)).max() <= 2e-6
