"""Host-side checks of the C-ABI library: it loads, exports every entry point
declared in include/nlos.h, validates arguments, and builds the R_z / R_t^{-1}
index tables and the sampled-column list bit-exactly like the oracle."""

import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import lct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import build, nlos as mod
    build.build_library()
    mod.load()
    return mod


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nlos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nlos_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(nlos):
    lib = ctypes.CDLL(nlos.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in nlos.h but not exported"
    assert set(names) == set(nlos.exported_symbols())


@pytest.mark.parametrize("nt", [16, 64, 256, 512, 1024])
@pytest.mark.parametrize("rad", ["compensated", "raw"])
def test_tables_bit_exact_against_oracle(nlos, nt, rad):
    t = nlos.geometry_tables(8, 8, nt, 32e-12, radiometry=rad)
    i0, w0, w1, g = lct.rz_table(nt)
    assert np.array_equal(t["rz_i0"], i0.astype(np.int32))
    assert np.array_equal(t["rz_w"][:, 0], w0.astype(np.float32))
    assert np.array_equal(t["rz_w"][:, 1], w1.astype(np.float32))
    assert np.array_equal(t["rz_w"][:, 2], g.astype(np.float32))
    k0, v0, v1, wt = lct.rt_table(nt, rad)
    assert np.array_equal(t["rt_k0"], k0.astype(np.int32))
    assert np.array_equal(t["rt_w"][:, 0], v0.astype(np.float32))
    assert np.array_equal(t["rt_w"][:, 1], v1.astype(np.float32))
    assert np.array_equal(t["rt_w"][:, 2], wt.astype(np.float32))


@pytest.mark.parametrize("kind", ["stride2", "stride4", "random", "single", "full"])
def test_sampled_columns_bit_exact(nlos, kind):
    n = 32
    if kind == "stride2":
        m = synth.stride_mask(n, n, 2)
    elif kind == "stride4":
        m = synth.stride_mask(n, n, 4)
    elif kind == "random":
        m = synth.random_mask(n, n, 0.25, 7)
    elif kind == "single":
        m = np.zeros((n, n), np.uint8)
        m[31, 0] = 1
    else:
        m = None
    t = nlos.geometry_tables(n, n, 64, 16e-12, mask=m)
    want = lct.sampled_columns(np.ones((n, n), np.uint8) if m is None else m)
    assert np.array_equal(t["cols"], want)


def test_invalid_geometry_is_rejected(nlos):
    for bad in [dict(nx=12, ny=12, nt=64), dict(nx=8, ny=16, nt=64), dict(nx=256, ny=256, nt=64),
                dict(nx=8, ny=8, nt=2048), dict(nx=8, ny=8, nt=8)]:
        with pytest.raises(nlos.NlosError) as e:
            nlos.geometry_tables(bad["nx"], bad["ny"], bad["nt"], 16e-12)
        assert e.value.status == -1
    with pytest.raises(nlos.NlosError):
        nlos.geometry_tables(8, 8, 64, -1.0)
    with pytest.raises(nlos.NlosError):
        nlos.geometry_tables(8, 8, 64, 16e-12, mask=np.zeros((8, 8), np.uint8))
    assert "mask" in nlos.last_error()


def test_params_default_match_paper(nlos):
    from tests.test_oracle_admm import _golden_params
    gp = _golden_params()
    p1, p2 = nlos.params_default(1), nlos.params_default(2)
    assert (p1.a, p1.b, p1.mu, p1.iters) == (gp["alg1_a_8x8"], gp["alg1_b_8x8"], gp["alg1_mu"], gp["alg1_tmax"])
    assert (p2.mu1, p2.mu2, p2.mu3, p2.iters) == (gp["alg2_mu1"], gp["alg2_mu2"], gp["alg2_mu3"], gp["alg2_tmax"])
    assert (p2.lambda_, p2.a_u, p2.b_u, p2.a_tau, p2.b_tau) == (
        gp["alg2_lambda_8x8"], gp["alg2_a_u_8x8"], gp["alg2_b_u_8x8"], gp["alg2_a_tau_8x8"], gp["alg2_b_tau_8x8"])
    with pytest.raises(nlos.NlosError):
        nlos.params_default(3)


def test_midpoint_conversion_validates_before_any_device_work(nlos):
    # every rejection happens on the host, before a launch: no GPU is needed
    buf_a, buf_b = 1 << 20, 1 << 30          # fake, 16-byte aligned, disjoint device addresses
    bad = [
        dict(nx=8, ny=8, nt=60),              # nt not a power of two
        dict(nx=6, ny=8, nt=64),              # nx not a power of two
        dict(nx=8, ny=8, nt=4096),            # nt above 2048
        dict(bin_width_s=0.0), dict(bin_width_s=float("inf")), dict(wall_width_m=-1.0),
        dict(laser=(float("nan"), 0.0)),
        dict(src=0), dict(dst=buf_a + 4),     # null input; output overlapping the input
        dict(dst=buf_b + 2),                  # misaligned output
    ]
    for b in bad:
        a = dict(nx=8, ny=8, nt=64, bin_width_s=32e-12, wall_width_m=1.0, laser=(0.0, 0.0), src=buf_a, dst=buf_b)
        a.update(b)
        with pytest.raises(nlos.NlosError) as e:
            nlos.midpoint_confocal(a["nx"], a["ny"], a["nt"], a["bin_width_s"], a["wall_width_m"], a["laser"],
                                   a["src"], a["dst"])
        assert e.value.status == -1, b


def test_server_prepare_validates_arguments(nlos):
    # argument checks of nlos_server_prepare need no device either
    lib = nlos.load()
    p = nlos.params_default(1)
    g, _keep = nlos._geometry(8, 8, 64, 32e-12, 1.0, "compensated", None)
    assert lib.nlos_server_prepare(None, ctypes.byref(g), ctypes.byref(p), 1, 1.0, None) == -1
