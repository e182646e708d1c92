"""CPU checks of the Python binding's argument validation: the C ABI takes
bare device pointers, so every array is checked (type, size, layout, device)
before a pointer is handed over; a bad one raises FlosicError(ARG) and
nothing reaches the library."""
import numpy as np
import pytest
import torch

from paper_2108_01186_gb300 import flosic as F


class _Ctx:
    """Stand-in with the attributes the checks read (no device work)."""
    device = torch.device("cuda", 0)


@pytest.mark.parametrize("t", [torch.zeros(8, dtype=torch.float64),            # host memory
                               np.zeros(8),                                      # not a tensor
                               torch.zeros(8, dtype=torch.float32),            # wrong type
                               torch.zeros(9, dtype=torch.float64),            # wrong size
                               torch.zeros(16, dtype=torch.float64)[::2]])     # not contiguous
def test_context_arrays_are_checked(t):
    with pytest.raises(F.FlosicError) as e:
        F.Context._req(_Ctx(), t, 8, "psi")
    assert e.value.code == F.FLOSIC_ERR_ARG


def test_noalloc_arrays_are_checked_before_any_call():
    F.load_library()
    grid = (4, 4, 4, 0.5, (0.0, 0.0, 0.0))
    phi = torch.zeros(2 * 64, dtype=torch.float64)
    for args in [(phi, phi),                                   # host memory
                 (np.zeros(128), phi),                         # not a tensor
                 (torch.zeros(100, dtype=torch.float64), phi)]:  # not a whole number of grids
        with pytest.raises(F.FlosicError) as e:
            F.orbital_poisson_noalloc(grid, *args)
        assert e.value.code == F.FLOSIC_ERR_ARG
