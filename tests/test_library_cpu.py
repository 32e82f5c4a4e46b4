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


def _harmonic_matrix(H):
    k = H.shape[1]
    Hk = H[:k, :k].copy()
    e = np.zeros(k)
    e[-1] = 1.0
    Hk[:, -1] += H[k, k - 1] ** 2 * np.linalg.solve(Hk.T, e)
    return Hk


def test_hessenberg_eigvals_of_perturbed_degree40_harmonic_matrices():
    """The degree-40 harmonic Ritz matrix of a convection-diffusion system (last column far larger
    than the rest) under 1e-13 relative perturbations -- rounding-level differences like those
    between two Arnoldi runs.  The unbalanced QR iteration failed to converge on most of them."""
    from oracle import gmres as og
    A, _, start = synth.workload_controller(50019, 128, 512)
    _, H, k = og.arnoldi(A, start, 41)
    H = np.asarray(H)
    rng = np.random.default_rng(0)
    for _ in range(200):
        M = _harmonic_matrix(H * (1.0 + 1e-13 * rng.normal(size=H.shape)))
        ev = g.hessenberg_eigvals(M)
        ref = np.linalg.eigvals(M)
        for z in ref:
            assert np.min(np.abs(ev - z)) <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("seed", range(4))
def test_hessenberg_eigvals_badly_scaled(seed):
    rng = np.random.default_rng(seed)
    k = 60
    H = np.triu(rng.normal(size=(k, k)), -1) * np.exp(3 * rng.normal(size=(k, k)))
    ev = g.hessenberg_eigvals(H)
    ref = np.linalg.eigvals(H)
    assert np.allclose(np.sort(np.abs(ev)), np.sort(np.abs(ref)), rtol=1e-6,
                       atol=1e-9 * np.abs(ref).max())


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding passes through the C ABI has the size and field offsets the
    header gives it (a C program compiled against include/gmresb3.h prints them)."""
    import ctypes
    import shutil
    import subprocess
    import paper_2105_07544_b300 as g
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"gmres_csr_t": g.CsrC, "gmres_precisions_t": g.PrecC, "gmres_params_t": g.ParamsC,
             "gmres_tuning_t": g.TuningC, "gmres_batch_tuning_t": g.BatchTuningC,
             "gmres_stats_t": g.StatsC, "gmres_suggestion_t": g.SuggestionC,
             "gmres_batch_stats_t": g.BatchStatsC}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gmresb3.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]) if len(l.split()) == 3 else None: int(l.split()[-1])
           for l in out if l.strip()}
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
