"""The binding's argument checks, on the CPU: state tensors that would hand the library
an invalid pointer or a short buffer (host memory, the wrong dtype, fewer cells than
requested, a Y layout other than [S, ld] planes with contiguous rows, status arrays of
the wrong type) are refused with CHEM_ERR_INVALID before anything reaches a kernel."""
import pytest
import torch

from paper_2506_02602_gb300 import chem


def _state(n):
    f = lambda *s: torch.zeros(*s, dtype=torch.float64)
    return f(n), f(n), f(9, n), f(n)


def test_host_tensors_are_refused():
    rho, e, Y, T = _state(8)
    with pytest.raises(chem.ChemError) as ei:
        chem._check_cells(8, rho, e, Y, T)
    assert ei.value.code == chem.ERR_INVALID and "CUDA" in str(ei.value)


def test_each_check_names_the_offending_argument(monkeypatch):
    # stand in for the CUDA-placement test so that the remaining checks are reached here
    def f64_only(name, t, n=None):
        if t.dtype != torch.float64:
            raise chem.ChemError(chem.ERR_INVALID, f"{name} must be a float64 CUDA tensor")
    monkeypatch.setattr(chem, "_check_f64_cuda", f64_only)
    rho, e, Y, T = _state(8)
    chem._check_cells(8, rho, e, Y, T)  # consistent arguments pass
    with pytest.raises(chem.ChemError, match="rho must be"):
        chem._check_cells(8, rho.float(), e, Y, T)
    with pytest.raises(chem.ChemError, match="T has 7 < 8"):
        chem._check_cells(8, rho, e, Y, T[:7])
    with pytest.raises(chem.ChemError, match="Y must be"):
        chem._check_cells(8, rho, e, Y.t().contiguous().t(), T)  # columns contiguous, not rows
    with pytest.raises(chem.ChemError, match="Y must be"):
        chem._check_cells(8, rho, e, Y[:, :7], T)                 # fewer cells than requested
    with pytest.raises(chem.ChemError, match="ncells < 0"):
        chem._check_cells(-1, rho, e, Y, T)
    with pytest.raises(chem.ChemError, match="status"):
        chem._check_cells(8, rho, e, Y, T, status=torch.zeros(8, dtype=torch.int64))
    with pytest.raises(chem.ChemError) as ei:
        chem._check_cells(8, rho, e, Y, T, nsteps=torch.zeros(8, dtype=torch.int32))  # host int32
    assert ei.value.code == chem.ERR_INVALID
