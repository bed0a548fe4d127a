"""Host side of the Nesterov placer (no GPU): the 3D mixed-size
preconditioner of eq. improved-precond on hand-made cases, the torch
statement the device loop is tested against."""
import pytest

torch = pytest.importorskip("torch")

from paper_2403_09070_gb300.nesterov import preconditioner  # noqa: E402


def test_preconditioner_hand_cases():
    # H = max(1, |E_i| + lambda q_i) for macros, max(1, lambda q_i) otherwise
    pins = torch.tensor([0.0, 5.0, 0.0, 3.0, 200.0], dtype=torch.float64)
    mac = torch.tensor([False, True, True, False, False])
    q = torch.tensor([10.0, 10.0, 10.0, 1e4, 1e4], dtype=torch.float64)
    H = preconditioner(pins, mac, q, 0.01)
    assert H.tolist() == pytest.approx([1.0, 5.1, 1.0, 100.0, 100.0])
    # the pin count enters for macros only, and nothing falls below 1
    H0 = preconditioner(pins, mac, q, 0.0)
    assert H0.tolist() == pytest.approx([1.0, 5.0, 1.0, 1.0, 1.0])
