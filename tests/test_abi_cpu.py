"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function that include/rpa.h declares, validates parameters, and
its host-only quadrature routine agrees with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as o
from paper_1307_8052_gb300 import binding as b
from paper_1307_8052_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return b.load()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "rpa.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rpa_[A-Za-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert "rpa_chi0" in names and "rpa_energy" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(b.SIGNATURES), "binding signatures out of step with the header"


def test_header_constants_match_the_binding():
    """Every enumerator and numeric macro of include/rpa.h (status codes,
    precision modes, tuning parameters, profile stage count) has the same value
    in the Python binding, so a knob added on one side cannot drift."""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "rpa.h")).read(), flags=re.S)
    consts = re.findall(r"\b(RPA_[A-Z0-9_]+)\s*=\s*(\d+)", txt)
    consts += re.findall(r"#define\s+(RPA_[A-Z0-9_]+)\s+(\d+)", txt)
    assert len(consts) >= 20
    for name, value in consts:
        assert getattr(b, name, None) == int(value), name


def test_gauss_legendre_matches_oracle(lib):
    for n in (1, 2, 8, 16, 33):
        for omega0 in (1.0, 0.4, 2.5):
            om, W = b.rpa_gauss_legendre(n, omega0)
            omr, Wr = o.frequency_grid(n, omega0)
            assert np.allclose(om, omr, rtol=1e-13, atol=0)
            assert np.allclose(W, Wr, rtol=1e-12, atol=0)
    with pytest.raises(b.RpaError) as e:
        b.rpa_gauss_legendre(0)
    assert e.value.status == b.RPA_ERR_ARG


def test_create_rejects_bad_parameters(lib):
    for kw in ({"grid": (1, 8, 8)}, {"ecut_chi": -1.0}, {"nk_bz": 0}, {"precision": 7},
               {"cell": np.zeros((3, 3))}):
        args = dict(cell=np.eye(3) * 5, grid=(8, 8, 8), ecut_chi=1.0)
        args.update(kw)
        with pytest.raises(b.RpaError) as e:
            b.rpa_create(**args)
        assert e.value.status == b.RPA_ERR_ARG


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(b.RpaError) as e:
        b.rpa_create(np.eye(3) * 5, (8, 8, 8), 1.0)
    assert e.value.status == b.RPA_ERR_CUDA
