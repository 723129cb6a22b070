"""The CUDA path's exponential- and power-cone projections (compiled for the
host from the same header the kernels use) against the oracle, on the CPU."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import cones

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("hostcones") / "hostcones.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           os.path.join(HERE, "host_cones.cu"), "-o", str(out)])
    return ctypes.CDLL(str(out))


def points(seed, count):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((count, 3)) * rng.uniform(0.1, 5, size=(count, 1))
    k = count // 5
    V[:k] *= 10.0 ** rng.uniform(-6, 3, size=(k, 3))       # mixed magnitudes
    return V


@pytest.mark.parametrize("dual", [0, 1])
def test_exp_projection_matches_oracle(lib, dual):
    V = points(10 + dual, 6000)
    out = np.zeros_like(V)
    lib.host_proj_exp(V.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p), len(V), dual)
    ref = np.array([cones.proj_exp_dual(v) if dual else cones.proj_exp(v) for v in V])
    err = np.linalg.norm(out - ref, axis=1) / np.maximum(1.0, np.linalg.norm(V, axis=1))
    assert err.max() <= 1e-12, (V[np.argmax(err)], out[np.argmax(err)], ref[np.argmax(err)])


@pytest.mark.parametrize("dual", [0, 1])
def test_exp_projection_fp32_matches_oracle(lib, dual):
    """The FP32 projection of the mixed-precision iteration, on FP32 inputs,
    within a few FP32 ulps (relative to ||v||) of the FP64 oracle's projection
    of the same inputs."""
    V = points(20 + dual, 6000).astype(np.float32)
    out = np.zeros_like(V)
    lib.host_proj_exp_f(V.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p), len(V), dual)
    Vd = V.astype(np.float64)
    ref = np.array([cones.proj_exp_dual(v) if dual else cones.proj_exp(v) for v in Vd])
    err = np.linalg.norm(out - ref, axis=1) / np.linalg.norm(Vd, axis=1)
    assert err.max() <= 2e-5, (Vd[np.argmax(err)], out[np.argmax(err)], ref[np.argmax(err)], err.max())
    assert np.median(err) <= 1e-6


def pow_points(seed, count):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((count, 3)) * rng.uniform(0.1, 5, size=(count, 1))
    k = count // 5
    V[:k] *= 10.0 ** rng.uniform(-6, 3, size=(k, 3))
    A = rng.uniform(0.02, 0.98, size=count)
    return V, A


@pytest.mark.parametrize("dual", [0, 1])
def test_pow_projection_matches_oracle(lib, dual):
    V, A = pow_points(30 + dual, 6000)
    out = np.zeros_like(V)
    lib.host_proj_pow(V.ctypes.data_as(ctypes.c_void_p), A.ctypes.data_as(ctypes.c_void_p),
                      out.ctypes.data_as(ctypes.c_void_p), len(V), dual)
    ref = np.array([cones.proj_pow_dual(v, a) if dual else cones.proj_pow(v, a) for v, a in zip(V, A)])
    err = np.linalg.norm(out - ref, axis=1) / np.maximum(1.0, np.linalg.norm(V, axis=1))
    assert err.max() <= 1e-12, (V[np.argmax(err)], A[np.argmax(err)], out[np.argmax(err)], ref[np.argmax(err)])


@pytest.mark.parametrize("dual", [0, 1])
def test_pow_projection_fp32_matches_oracle(lib, dual):
    """The FP32 power-cone projection (the mixed-precision iteration's) on
    FP32 inputs, within a few FP32 ulps (relative to ||v||) of the oracle."""
    V, A = pow_points(40 + dual, 6000)
    V = V.astype(np.float32)
    A = A.astype(np.float32)
    out = np.zeros_like(V)
    lib.host_proj_pow_f(V.ctypes.data_as(ctypes.c_void_p), A.ctypes.data_as(ctypes.c_void_p),
                        out.ctypes.data_as(ctypes.c_void_p), len(V), dual)
    Vd, Ad = V.astype(np.float64), A.astype(np.float64)
    ref = np.array([cones.proj_pow_dual(v, a) if dual else cones.proj_pow(v, a) for v, a in zip(Vd, Ad)])
    err = np.linalg.norm(out - ref, axis=1) / np.linalg.norm(Vd, axis=1)
    assert err.max() <= 2e-5, (Vd[np.argmax(err)], Ad[np.argmax(err)], out[np.argmax(err)], ref[np.argmax(err)])
    assert np.median(err) <= 1e-6
