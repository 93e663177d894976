"""The seeded input recipes (chem_inputs.workloads), on the CPU: the sizes, classes and
ranges the benchmark and its documentation quote for each workload."""
import numpy as np

from chem_inputs import workloads as W

ATM = W.ATM


def _mass_fractions_ok(Y):
    assert np.all(Y >= 0.0) and np.allclose(Y.sum(axis=0), 1.0, rtol=0, atol=1e-12)


def test_reactors():
    r = W.reactors(4096, seed=0)
    assert r["T"].size == 4096 and r["Y"].shape == (9, 4096)
    assert r["phi"].min() >= 0.5 and r["phi"].max() <= 2.0
    assert r["T"].min() >= 1000.0 and r["T"].max() <= 2000.0
    assert r["p"].min() >= 0.5 * ATM and r["p"].max() <= 5.0 * ATM
    _mass_fractions_ok(r["Y"])
    # fresh hydrogen-air without radicals; the same seed gives the same states
    assert np.all(r["Y"][W.IDX["H"]] == 0.0) and np.all(r["Y"][W.IDX["OH"]] == 0.0)
    assert np.array_equal(W.reactors(4096, seed=0)["T"], r["T"])


def test_amr_batch_sizes_classes_and_levels():
    b = W.amr_batch()
    off, nsub = b["box_offset"], b["box_nsub"]
    ncell = np.diff(off)
    assert off[0] == 0 and off[-1] == b["T"].size == 3_457_024        # the batch's realised cells
    assert int((ncell * nsub).sum()) == 7_991_808                       # cell-substeps
    assert set(np.round(np.cbrt(ncell)).astype(int)) <= {8, 16, 24, 32}
    assert np.array_equal(b["box_level"], np.arange(256) % 3)
    assert np.array_equal(nsub, 2 ** b["box_level"]) and np.allclose(b["box_dt"], 1e-7 / nsub)
    frac = np.bincount(b["cls"], minlength=3) / b["cls"].size
    assert abs(frac[0] - 0.90) < 0.005 and abs(frac[1] - 0.08) < 0.005 and abs(frac[2] - 0.02) < 0.005
    _mass_fractions_ok(b["Y"])
    front = b["cls"] == 2
    assert np.all(b["Y"][W.IDX["H"], front] > 4e-5) and np.all(b["T"][front] >= 1500.0)


def test_detonation_slice_regions():
    nx, ny = 1024, 4
    d = W.detonation_slice(nx, ny, seed=1)
    T = d["T"].reshape(ny, nx)
    assert d["Y"].shape == (9, nx * ny)
    # pre-shock quarter at 300 K (+-2 % noise), burnt end at 2900 K
    assert np.all(np.abs(T[:, : nx // 4] / 300.0 - 1.0) <= 0.02 + 1e-12)
    assert np.all(np.abs(T[:, -10:] / 2900.0 - 1.0) <= 0.02 + 1e-12)
    # the induction zone rises from 1200 to 1600 K
    assert 1150 < T[:, nx // 4 + 2].mean() < 1260 and 1500 < T[:, int(0.45 * nx) - 2].mean() < 1650
    _mass_fractions_ok(d["Y"])


def test_eq27_profile():
    for alpha in (1.0, 0.1):
        d = W.eq27_profile(alpha)
        assert d["T"].size == 65_536
        A = 50.0 / alpha
        assert d["T"].min() >= 1000.0 - A and d["T"].max() <= 1600.0 + A
        X = d["Y"][:, 0] / np.array(W._W())
        X /= X.sum()
        assert np.allclose(X[[W.IDX["H2"], W.IDX["O2"], W.IDX["N2"]]], [0.1, 0.2, 0.7])
        # T varies along y only: every x-z column repeats the same profile
        T = d["T"].reshape(256, 256)
        assert np.all(T == T[0])
