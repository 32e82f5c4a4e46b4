"""Host-side checks of the C-ABI library (no GPU): it loads, exports every declared symbol, its
host eigenvalue routine matches LAPACK, and compute entry points fail loudly without a GPU."""
import os
import re

import numpy as np
import pytest
import torch

import paper_2105_07544_b300 as g
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "gmresb3.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gmres_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = g.load()
    syms = _declared_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) <= set(g._SIGS), set(syms) - set(g._SIGS)


def test_status_strings():
    for code in (0, -1, -2, -3, -4, 1, 2, 3, 4, 5):
        assert g.status_string(code) != "unknown status"


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7, 26, 41, 80])
def test_hessenberg_eigvals_match_lapack(k):
    rng = np.random.default_rng(k)
    H = np.triu(rng.standard_normal((k, k)), -1)
    ev = g.hessenberg_eigvals(H)
    ref = np.linalg.eigvals(H)
    assert np.max(np.abs(np.sort_complex(ev) - np.sort_complex(ref))) <= 1e-10 * max(1, np.abs(ref).max())


def test_hessenberg_eigvals_arnoldi_of_convdiff():
    from oracle import gmres as og
    A = synth.convdiff2d(30, 0.5, 100.0)
    V, H, k = og.arnoldi(A, synth.uniform(A.n, 0), 40)
    Hk = H[:40, :40]
    ev = g.hessenberg_eigvals(Hk)
    ref = np.linalg.eigvals(Hk)
    assert np.max(np.abs(np.sort_complex(ev) - np.sort_complex(ref))) <= 1e-9 * np.abs(ref).max()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_create_without_gpu_fails_loudly():
    A = synth.laplace2d(8)
    with pytest.raises(g.GmresError) as e:
        g.Solver(A, m=10)
    assert e.value.code == -3
