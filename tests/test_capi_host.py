"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point that include/lks.h declares, validates descriptors, and its
generalized-inverse edge maps equal the paper's closed form and the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import inputs
from oracle import oracle as O
from paper_2411_03090_gb300 import lks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _declared():
    src = open(os.path.join(ROOT, "include", "lks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:lks|alks)_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = lks.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(lks.EXPORTS)


def test_status_strings():
    L = lks.load()
    for s in range(8):
        assert L.lks_status_string(s)


def _moments(f):
    return np.array([W @ f, W @ (CX * f), W @ (CY * f), W @ (CX * CX * f), W @ (CX * CY * f),
                     W @ (CY * CY * f)])


@pytest.mark.parametrize("A", [-0.6675, 0.17625, 0.3])
def test_bottom_face_map_is_eq_ftilde(A):
    """Moments of the bottom-face fill equal those of Eq. (ftilde) (Sec. 2.5)."""
    M = lks.edge_moment_map(A, 3)[:, :9]
    rng = np.random.default_rng(0)
    f = rng.standard_normal(9)
    f[[4, 7, 8]] = 0.0
    full = f.copy()
    full[4] = (f[2] + f[5] + f[6]) / 3
    full[7] = (4 * f[2] + 7 * f[5] + f[6]) / 12
    full[8] = (4 * f[2] + f[5] + 7 * f[6]) / 12
    np.testing.assert_allclose(M @ f, _moments(full), atol=1e-14)


@pytest.mark.parametrize("cls,n,pressure", [(0, (-1, 0), 0), (1, (1, 0), 1), (2, (1, 0), 0),
                                            (3, (0, -1), 0), (4, (0, 1), 0), (5, (-1, -1), 0),
                                            (6, (1, -1), 0), (7, (-1, 1), 0), (8, (1, 1), 0)])
def test_edge_maps_match_oracle(cls, n, pressure):
    A = -0.2
    M = lks.edge_moment_map(A, cls)
    rng = np.random.default_rng(cls)
    unknown = np.array([1 if (CX[k] * n[0] > 0 or CY[k] * n[1] > 0) else 0 for k in range(9)])
    f = rng.standard_normal(9) * (1 - unknown)
    kT = 0.37
    full, _ = O.bc_flow(n, pressure, A, f, unknown, kT=kT)
    np.testing.assert_allclose(M[:, :9] @ f + M[:, 9] * kT, _moments(full), atol=1e-13)


def test_descriptor_validation():
    pb = inputs.config1()
    d = lks.make_desc(pb)
    assert lks.workspace_size(d) > 0
    for field, val in (("nx", 3), ("real_type", 7), ("nu", 0.9), ("version", 99), ("n_steps", 0)):
        bad = lks.make_desc(pb)
        setattr(bad, field, val)
        with pytest.raises(lks.LKSError) as e:
            lks.workspace_size(bad)
        assert e.value.status == 1
    bad = lks.make_desc(pb)
    bad.reserved[3] = 1
    with pytest.raises(lks.LKSError):
        lks.workspace_size(bad)


def test_workspace_grows_with_checkpoint_storage():
    p3 = inputs.config3().with_(nx=64, ny=32, n_steps=1000)
    plain = lks.workspace_size(lks.make_desc(p3, checkpoint_every=0))
    ck = lks.workspace_size(lks.make_desc(p3, checkpoint_every=100, snapshot="bf16"))
    assert ck < plain


def test_create_rejects_bad_workspace_without_gpu_work():
    L = lks.load()
    d = lks.make_desc(inputs.config1())
    h = C.c_void_p()
    st = L.lks_create(C.byref(d), None, C.c_size_t(16), None, C.byref(h))
    assert st == 2 and not h.value
