"""Host-side parts of the learned min-sum recipe: checkpoint round trip, the stored table
format and the BLER-crossing interpolation (no GPU)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_05534_gb300 import learned
from paper_2009_05534_gb300.train_learned import ebn0_at, load_table, save_table


def test_checkpoint_round_trip(tmp_path):
    p = torch.full((3, 4, 2), 0.75, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3)
    for _ in range(3):
        opt.zero_grad()
        (p * torch.arange(24.0).reshape(3, 4, 2)).sum().backward()
        opt.step()
    path = tmp_path / "ck.pt"
    learned.save_checkpoint(path, p, opt, 3, [0.5, 0.4, 0.3])
    ck = learned.load_checkpoint(path)
    assert ck["step"] == 3 and ck["loss"] == [0.5, 0.4, 0.3]
    assert torch.equal(ck["params"], p.detach())
    q = torch.zeros((3, 4, 2), requires_grad=True)
    opt2 = torch.optim.Adam([q], lr=1e-3)
    opt2.load_state_dict(ck["adam"])
    st1 = opt.state_dict()["state"][0]
    st2 = opt2.state_dict()["state"][0]
    assert torch.equal(st1["exp_avg"], st2["exp_avg"])
    assert torch.equal(st1["exp_avg_sq"], st2["exp_avg_sq"])


def test_table_json_round_trip(tmp_path):
    t = np.random.default_rng(0).random((10, 42, 2)).astype(np.float32)
    path = tmp_path / "t.json"
    save_table(path, t, {"T": 10, "n_rows": 42})
    t2, meta = load_table(path)
    assert np.array_equal(t, t2)
    assert meta["shape"] == [10, 42, 2] and meta["T"] == 10


def test_ebn0_at_interpolates_log_linearly():
    grid = [1.0, 2.0, 3.0]
    assert ebn0_at(grid, [1.0, 0.1, 0.001], 1e-2) == pytest.approx(2.5)
    assert ebn0_at(grid, [0.005, 0.001, 0.0], 1e-2) == 1.0
    assert ebn0_at(grid, [1.0, 0.5, 0.2], 1e-2) is None
    assert ebn0_at(grid, [1.0, 0.5, 0.0], 1e-2) == 3.0
    b = ebn0_at([0.0, 1.0], [0.1, 0.0001], 1e-2)
    assert b == pytest.approx(1.0 / 3.0)
    assert math.isfinite(b)


def test_stored_tables_are_well_formed():
    import glob
    import os
    from paper_2009_05534_gb300.train_learned import TABLE_DIR
    for path in glob.glob(os.path.join(TABLE_DIR, "*.json")):
        t, meta = load_table(path)
        assert t.shape == (meta["T"], meta["n_rows"], 2)
        assert np.isfinite(t).all()
        assert (t[..., 0] > 0).all()          # a positive scale keeps the min-sum sign rule
