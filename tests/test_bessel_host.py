"""The K_nu quadrature of the FP64 paths (trapezoidal rule on
K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt, DLMF 10.32.9) and the
general-nu Matern correlation built on it (Eq. maternkernel), compiled for the
host from the same header the kernels include, against scipy's K_nu (Amos'
algorithm, an independent implementation) and the closed forms at
half-integer nu.
"""
import ctypes
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest
from scipy.special import gamma, kv

HERE = Path(__file__).parent


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("bessel") / "libbessel_host.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    str(HERE / "native" / "bessel_host.cpp"), "-o", str(out)], check=True)
    L = ctypes.CDLL(str(out))
    for f in (L.sbv_test_bessel_k, L.sbv_test_matern_general):
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_double, ctypes.c_double]
    return L


def test_bessel_k_matches_scipy_over_orders_and_arguments(lib):
    worst = 0.0
    for nu in [0.0, 0.3, 0.5, 1.0, 1.7, 2.5, 4.0, 7.5, 12.25, 19.5, 20.0]:
        for x in np.logspace(-8, np.log10(700.0), 60):
            ref = kv(nu, x)
            if not np.isfinite(ref) or ref == 0.0 or ref > 1e300:
                continue
            got = lib.sbv_test_bessel_k(nu, x)
            worst = max(worst, abs(got - ref) / ref)
    # the header's stated bound is 1e-12 for nu <= 20
    assert worst < 1e-12, worst


def test_matern_general_reduces_to_closed_forms(lib):
    r = np.concatenate([np.logspace(-6, -1, 20), np.linspace(0.1, 40.0, 80)])
    closed = {
        1: lambda r: np.exp(-r),
        3: lambda r: (1 + r) * np.exp(-r),
        5: lambda r: (1 + r + r * r / 3) * np.exp(-r),
        7: lambda r: (1 + r + 2 * r * r / 5 + r ** 3 / 15) * np.exp(-r),
    }
    for nu2, f in closed.items():
        got = np.array([lib.sbv_test_matern_general(v, nu2 / 2) for v in r])
        np.testing.assert_allclose(got, f(r), rtol=2e-12, atol=1e-300)


def test_matern_general_matches_its_definition(lib):
    for nu in [1.0, 1.5, 2.0, 3.3, 4.5, 9.0, 17.5]:
        for r in np.logspace(-4, np.log10(60.0), 40):
            ref = 2.0 ** (1 - nu) / gamma(nu) * r ** nu * kv(nu, r)
            got = lib.sbv_test_matern_general(r, nu)
            assert abs(got - ref) <= 1e-12 * max(ref, 1e-300), (nu, r, got, ref)
    # below the cut-off the correlation is taken as 1 (its limit at r = 0)
    assert lib.sbv_test_matern_general(0.0, 2.0) == 1.0
