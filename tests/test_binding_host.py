"""Host-side logic of the Python binding that needs no GPU: the boundary
layout's size, the grid screen that decides which arrays are size-checked,
and the size checks themselves (on CPU tensors)."""
import pytest

torch = pytest.importorskip("torch")

from paper_math_9809043_gb300 import msrcg as M  # noqa: E402
from paper_math_9809043_gb300 import problems as P  # noqa: E402


@pytest.mark.parametrize("dim,n", [(2, (7, 5)), (2, (1, 1)), (3, (4, 3, 2)), (3, (1, 1, 9))])
def test_boundary_face_count(dim, n):
    assert M.n_boundary_faces(dim, n) == P.n_boundary_faces(dim, n)
    bc, gD = P.standard_bc(dim, n)
    assert bc.size == gD.size == M.n_boundary_faces(dim, n)


def test_grid_screen():
    assert M._valid_grid(2, (8, 8)) and M._valid_grid(3, (2, 3, 4)) and M._valid_grid(2, (1, 1))
    assert not M._valid_grid(2, (0, 8)) and not M._valid_grid(4, (8, 8)) and not M._valid_grid(3, (8, 8))


def test_size_checks_on_host_tensors():
    cpu = torch.device("cpu")
    t = M._dev([1.0, 2.0, 3.0], torch.float64, cpu, 3, "b")
    assert t.dtype == torch.float64 and t.numel() == 3
    with pytest.raises(ValueError):
        M._dev([1.0, 2.0], torch.float64, cpu, 3, "b")
    x = torch.empty(4, dtype=torch.float64)
    assert M._out(x, torch.float64, cpu, 4, "x") is x
    for bad in (torch.empty(5, dtype=torch.float64), torch.empty(4, dtype=torch.float32),
                torch.empty(8, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            M._out(bad, torch.float64, cpu, 4, "x")
    assert M._check_K(torch.ones(12, dtype=torch.float64), 2, 6) == 2
    assert M._check_K(torch.ones(6, dtype=torch.float64), 3, 6) == 1
    with pytest.raises(ValueError):
        M._check_K(torch.ones(7, dtype=torch.float64), 2, 6)
    with pytest.raises(ValueError):
        M._check_K(torch.ones(24, dtype=torch.float64), 3, 6)
