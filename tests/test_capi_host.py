"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, and its host-only logic (parameters, K, AUC) behaves.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wdad.h")


@pytest.fixture(scope="module")
def wl():
    from paper_1201_2025_gb300 import build, wdad
    build.build()
    return wdad


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wdad_[A-Za-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(wl):
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1201_2025_gb300", "libwdad.so"))
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params(wl):
    p = wl.wdad_default_params()
    assert (p.wavelet_taps, p.level, p.inner, p.outer, p.border, p.dwest_mode, p.precision) == (8, -1, 3, 11, 0, 0, 0)
    assert abs(p.loading - 1e-3) < 1e-9 and abs(p.cond_gate - 1e6) < 1 and abs(p.dwest_tau - 1e-6) < 1e-12


@pytest.mark.parametrize("L,level", [(224, -1), (188, -1), (189, -1), (128, -1), (4, -1), (3, -1), (224, 3), (1, 5)])
def test_query_K_matches_oracle_levels(wl, L, level):
    assert wl.wdad_query_K(L, 8, level) == oracle.dwt_levels(L, level)[1]


def test_query_K_rejects_bad_input(wl):
    assert wl.wdad_query_K(0, 8, -1) == -1
    assert wl.wdad_query_K(224, 7, -1) == -1   # odd filter length
    assert wl.wdad_query_K(224, 22, -1) == -1  # beyond db10
    assert wl.wdad_query_K(224, 0, -1) == -1
    assert wl.wdad_query_K(224, 8, -2) == -1
    assert wl.wdad_query_K(224, 6, -1) == wl.wdad_query_K(224, 8, -1)  # K does not depend on the filter


@pytest.mark.parametrize("taps", [2, 4, 6, 8, 10, 12, 14, 16, 18, 20])
def test_wavelet_filter_matches_oracle(wl, taps):
    # two independent constructions of Daubechies' filter (Laguerre here, Durand-Kerner in the
    # oracle); the oracle's is pinned to the published db4 / D4 values and the filter identities
    np.testing.assert_allclose(wl.wdad_wavelet_filter(taps), oracle.daub_filter(taps), rtol=0, atol=1e-12)


def test_wavelet_filter_published_values(wl):
    s3, r = np.sqrt(3.0), 4 * np.sqrt(2.0)
    np.testing.assert_allclose(wl.wdad_wavelet_filter(4), [(1 + s3) / r, (3 + s3) / r, (3 - s3) / r, (1 - s3) / r],
                               rtol=0, atol=1e-15)
    db4 = [0.2303778133088964, 0.7148465705529154, 0.6308807679298587, -0.0279837694168599,
           -0.1870348117190931, 0.0308413818355607, 0.0328830116668852, -0.0105974017850690]
    np.testing.assert_allclose(wl.wdad_wavelet_filter(8), db4, rtol=0, atol=1e-15)
    for bad in (0, 3, 22):
        with pytest.raises(wl.WdadError):
            wl.wdad_wavelet_filter(bad)


def test_null_handle_is_an_argument_error(wl):
    lib = wl.lib()
    p = wl.wdad_default_params()
    assert lib.wdad_detect(None, None, 4, 4, 224, 0, 1, ctypes.byref(p), None, None, None) == wl.WDAD_ERR_ARG
    assert lib.wdad_detect_sequence(None, 1, None, 4, 4, 224, 1, ctypes.byref(p), None, None, None) == wl.WDAD_ERR_ARG
    assert lib.wdad_destroy(None) == wl.WDAD_ERR_ARG


def test_auc_matches_oracle(wl):
    rng = np.random.default_rng(0)
    s = np.round(rng.standard_normal(20000), 2).astype(np.float32)
    s[::97] = np.nan
    m = (rng.uniform(size=s.size) < 0.05).astype(np.uint8)
    assert abs(wl.wdad_auc(s, m) - oracle.auc(s.astype(np.float64), m)) < 1e-12
    assert np.isnan(wl.wdad_auc(s, np.zeros_like(m)))


def test_binding_fails_loudly_without_the_library(monkeypatch):
    # no CPU fallback: without libwdad.so every call raises instead of computing elsewhere
    from paper_1201_2025_gb300 import wdad
    monkeypatch.setattr(wdad, "_lib", None)
    monkeypatch.setattr(wdad, "_SO", os.path.join(ROOT, "no_such_dir", "libwdad.so"))
    with pytest.raises(RuntimeError, match="missing"):
        wdad.lib()
    with pytest.raises(RuntimeError, match="missing"):
        wdad.wdad_query_K(224)
