"""The C ABI library loads and exports every symbol include/lb.h declares;
host-only calls work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np

import pytest

from tests.helpers import A_VDW, B_VDW, library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lb = library()
    lib = ctypes.CDLL(lb.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_coexistence_host_call_matches_oracle():
    from oracle import lb_oracle as O
    lb = library()
    for T in (0.30, 0.45, 0.50, 0.55, 0.56):
        rl, rg = lb.coexistence(A_VDW, B_VDW, T)
        orl, org = O.coexistence(A_VDW, B_VDW, T)
        assert abs(rl - orl) < 1e-12 * orl and abs(rg - org) < 1e-11 * org


def test_invalid_parameters_rejected_before_device_work():
    lb = library()
    bad = [dict(tau=0.5), dict(tau=0.3), dict(T=0.6), dict(kappa=0.0), dict(shape=(0, 4))]
    for b in bad:
        kw = dict(shape=(8, 8), a=A_VDW, b=B_VDW, T=0.55, kappa=0.01, tau=0.8)
        kw.update(b)
        with pytest.raises(lb.LBError) as e:
            lb.Context(0, kw["shape"], kw["a"], kw["b"], kw["T"], kw["kappa"], kw["tau"])
        assert e.value.status == 1
    with pytest.raises(lb.LBError):
        lb.Context(0, (8, 8, 2), A_VDW, B_VDW, 0.55, 0.01, 0.8)   # D2Q9 needs nz = 1
    with pytest.raises(lb.LBError):
        lb.coexistence(A_VDW, B_VDW, 8 * A_VDW / (27 * B_VDW))
    # site indices are 32-bit in the kernels: more than 2^31 - 1 sites is refused
    with pytest.raises(lb.LBError) as e:
        lb.Context(1, (1300, 1300, 1300), A_VDW, B_VDW, 0.55, 0.01, 0.8)
    assert e.value.status == 1 and "32-bit" in str(e.value)


def test_batch_limits_rejected_before_device_work():
    """A batch work item holds 12 bits of instance and 20 bits of tile: more than
    4096 instances or 2^20 tiles of 32 x 8 in one instance is refused."""
    lb = library()
    ok = dict(nx=32, ny=32, T=0.55, kappa=0.01, tau=1.0, radius=8.0)
    with pytest.raises(lb.LBError) as e:
        lb.Batch([dict(ok, nx=32768, ny=8200)], A_VDW, B_VDW)
    assert e.value.status == 1
    with pytest.raises(lb.LBError) as e:
        lb.Batch([ok] * 4097, A_VDW, B_VDW)
    assert e.value.status == 1


def test_missing_library_fails_loudly(tmp_path):
    from paper_0710_5470_gb300 import lb
    saved = lb._lib
    lb._lib = None
    try:
        with pytest.raises(RuntimeError):
            lb.load_library(str(tmp_path / "nope.so"))
    finally:
        lb._lib = saved


def test_fma_peak_arguments_rejected_before_device_work():
    lb = library()
    for args in ((2, 100), (0, 0), (1, (1 << 24) + 1)):
        with pytest.raises(lb.LBError) as e:
            lb.fma_peak(*args)
        assert e.value.status == 1


def test_params_hash_is_stable_and_sensitive():
    """lb_params_hash (host only): equal parameters give equal hashes; a change
    of any one parameter (lattice size, scheme, storage, a, b, T, kappa, tau,
    rho_ref) changes it; an invalid parameter set is rejected."""
    lb = library()
    base = dict(lattice=lb.D3Q19, shape=(16, 12, 8), a=A_VDW, b=B_VDW, T=0.55, kappa=0.01, tau=1.0,
                scheme=lb.FORCING, storage=lb.F16DEV, rho_ref=0.0)
    h0 = lb.params_hash(**base)
    assert h0 == lb.params_hash(**base)
    changes = [dict(shape=(16, 12, 9)), dict(shape=(18, 12, 8)), dict(scheme=lb.EQUILIBRIUM),
               dict(storage=lb.BF16DEV), dict(a=A_VDW * (1 + 1e-15)), dict(T=0.55 + 1e-12), dict(kappa=0.0101),
               dict(tau=0.9), dict(rho_ref=4.0), dict(lattice=lb.D2Q9, shape=(16, 12))]
    seen = {h0}
    for ch in changes:
        h = lb.params_hash(**dict(base, **ch))
        assert h not in seen, ch
        seen.add(h)
    with pytest.raises(lb.LBError):
        lb.params_hash(**dict(base, tau=0.4))


def test_binary_parameters_rejected_before_device_work():
    """lb_binary_create validates its parameters on the host (LB_EINVAL) before any CUDA call."""
    lb = library()
    ok = dict(A=-0.04, B=0.04, kappa=0.08, Gamma=1.0, tau=1.0, tau_phi=1.0)
    bad = [dict(tau=0.5), dict(tau_phi=0.4), dict(Gamma=0.0), dict(kappa=-1.0), dict(B=-0.1),
           dict(A=float("nan"))]
    for b in bad:
        kw = dict(ok)
        kw.update(b)
        with pytest.raises(lb.LBError) as e:
            lb.BinaryContext((16, 8), **kw)
        assert e.value.status == 1, b
    for shape, extra in (((0, 8), {}), ((8, 8), dict(scheme=2)), ((8, 8), dict(storage=3)),
                         ((9, 8), dict(storage=2)), ((8, 8, 4), dict(storage=2))):
        with pytest.raises(lb.LBError) as e:
            lb.BinaryContext(shape, **ok, **extra)
        assert e.value.status == 1


def test_population_bytes_host_only():
    """lb_population_bytes: 2 buffers x pitch (sites rounded up to 128) x bytes per site."""
    lb = library()
    per_site = {lb.F64: (8, 8), lb.F32: (4, 4), lb.F16DEV: (4, 2), lb.BF16DEV: (4, 2)}
    for lat, shape, q in ((lb.D2Q9, (37, 11), 9), (lb.D3Q19, (32, 8, 5), 19)):
        n = int(np.prod(shape))
        pitch = (n + 127) // 128 * 128
        for st, (b0, bi) in per_site.items():
            got = lb.population_bytes(lat, shape, A_VDW, B_VDW, 0.55, 0.01, 0.8, storage=st)
            assert got == 2 * pitch * (b0 + (q - 1) * bi), (lat, st)
    with pytest.raises(lb.LBError):
        lb.population_bytes(lb.D2Q9, (8, 8), A_VDW, B_VDW, 0.55, 0.01, 0.5)


def test_caller_buffer_checked_before_device_work():
    """lb_create_with_buffers refuses a NULL, unaligned or too small buffer on the host."""
    lb = library()
    need = lb.population_bytes(lb.D2Q9, (16, 8), A_VDW, B_VDW, 0.55, 0.01, 0.8)
    for ptr, nbytes in ((0, need), (256 * 1000 + 8, need), (256 * 1000, need - 1)):
        with pytest.raises(lb.LBError) as e:
            lb.Context(0, (16, 8), A_VDW, B_VDW, 0.55, 0.01, 0.8, buffer=(ptr, nbytes))
        assert e.value.status == 1
