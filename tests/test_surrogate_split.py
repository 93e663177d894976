"""The surrogate's data splits, on the CPU: whole trajectories go to one side of a split
(no trajectory contributes states to both training and validation or held-out cells),
the split is seeded, and drawn cells come only from the given set."""
import numpy as np
import torch

from paper_2506_02602_gb300 import surrogate


def _states(ntraj=200, per=7):
    traj = torch.arange(ntraj).repeat_interleave(per)
    n = traj.numel()
    g = torch.Generator().manual_seed(0)
    return {"traj": traj, "T": torch.rand(n, generator=g, dtype=torch.float64) * 1000 + 1000,
            "Y": torch.rand(9, n, generator=g, dtype=torch.float64), "rho": torch.ones(n, dtype=torch.float64)}


def test_split_keeps_trajectories_whole_and_is_seeded():
    st = _states()
    tr, held = surrogate.split_by_trajectory(st, 0.1, seed=3)
    a, b = set(tr["traj"].tolist()), set(held["traj"].tolist())
    assert a.isdisjoint(b) and a | b == set(range(200))
    assert tr["T"].numel() + held["T"].numel() == st["T"].numel()
    assert 5 <= len(b) <= 40                      # about 10 % of 200 trajectories
    assert tr["Y"].shape == (9, tr["T"].numel()) and tr["Y"].is_contiguous()
    tr2, held2 = surrogate.split_by_trajectory(st, 0.1, seed=3)
    assert torch.equal(held["traj"], held2["traj"])
    _, held3 = surrogate.split_by_trajectory(st, 0.1, seed=4)
    assert not torch.equal(held["traj"], held3["traj"])


def test_drawn_cells_come_from_the_set():
    st = _states()
    _, held = surrogate.split_by_trajectory(st, 0.1, seed=3)
    cells = surrogate.draw_cells(held, 1000, seed=5)
    assert cells["T"].numel() == 1000
    assert set(cells["traj"].tolist()) <= set(held["traj"].tolist())
    # every drawn cell is one of the set's states, all fields from the same state
    key = {(round(float(t), 9), int(j)) for t, j in zip(held["T"], held["traj"])}
    assert all((round(float(t), 9), int(j)) in key for t, j in zip(cells["T"], cells["traj"]))
    i = int(np.argmax(cells["T"].numpy()))
    k = int(torch.nonzero(held["T"] == cells["T"][i])[0])
    assert torch.equal(cells["Y"][:, i], held["Y"][:, k])
