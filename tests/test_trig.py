"""Accuracy of the FP32 sine/cosine of the Kalman step kernels (Cody-Waite reduction and
Taylor series), built for the host and checked against FP64 at 2 ulp."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def trig(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("trig") / "libtrig.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_2312_11728_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "trig_host.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    P = ctypes.POINTER(ctypes.c_float)

    def run(x):
        x = np.ascontiguousarray(x, np.float32)
        s, c = np.empty_like(x), np.empty_like(x)
        lib.trig_sweep(x.ctypes.data_as(P), s.ctypes.data_as(P), c.ctypes.data_as(P), ctypes.c_long(x.size))
        return s, c
    return run


def _ulp_err(got, exact):
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    return np.abs(got.astype(np.float64) - exact) / ulp


def _check(trig, x, bound=2.0):
    s, c = trig(x)
    xd = x.astype(np.float64)
    es, ec = _ulp_err(s, np.sin(xd)), _ulp_err(c, np.cos(xd))
    assert es.max() <= bound, (x[es.argmax()], es.max())
    assert ec.max() <= bound, (x[ec.argmax()], ec.max())


def test_dense_small_angles(trig):
    _check(trig, np.linspace(-8.0, 8.0, 2_000_001, dtype=np.float32))


def test_tiny_and_special(trig):
    x = np.array([0.0, -0.0, 1e-30, -1e-30, 1e-8, 1e-4, 0.5, 1.0, np.pi / 4], np.float32)
    _check(trig, x)
    s, c = trig(np.array([np.nan, np.inf], np.float32))
    assert np.isnan(s).all() and np.isnan(c).all()


def test_random_wide(trig):
    rng = np.random.default_rng(7)
    _check(trig, rng.uniform(-2.0 ** 15, 2.0 ** 15, 1_000_000).astype(np.float32))


def test_next_to_multiples_of_half_pi(trig):
    # the floats nearest to k*pi/2 and their neighbours, where the reduced argument is smallest
    k = np.arange(-4000, 4001, dtype=np.float64)
    base = (k * np.pi / 2).astype(np.float32)
    x = np.concatenate([base, np.nextafter(base, np.float32(np.inf)), np.nextafter(base, np.float32(-np.inf))])
    _check(trig, x)
