"""Winding number of the Larmor angle on the GPU against the oracle's definition, and the
coarsening driver end to end on a small case."""
import numpy as np
import pytest
import torch

from oracle import gpe_oracle as O
from paper_2310_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MEAN = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_03636_gb300 import binding
    return binding


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_winding_matches_oracle_ragged(B, dtype):
    shapes = [(256,), (8192,), (1024,), (256,)]
    b = B.GPEBatch(list(shapes), dtype=dtype, c1=-0.1, q=0.09, dt=0.04)
    b.init_noise(8, MEAN, 0.5)
    b.step(1500)
    nb, sd = b.layout()
    acc = torch.zeros(2 * sd, dtype=torch.float64, device="cuda")
    b.observables(acc, B.GPE_OBS_WINDING, 1)
    b.observables(acc, B.GPE_OBS_WINDING, 1)
    assert b.sync_status() == B.GPE_OK
    a = acc.cpu().numpy()
    assert np.all(a[:sd] == 0)
    got = B.unpack_winding(a[sd:], nb, len(shapes)) / 2
    ref = np.array([float(O.winding_number(torch.as_tensor(p.cpu().numpy().astype(np.complex128)))) for p in b.psi])
    np.testing.assert_allclose(got, ref, atol=1e-9)
    assert np.abs(got - np.round(got)).max() < 1e-6
    b.close()


def test_planted_winding(B):
    """psi_1 = a e^{2 pi i 3 x/L}, psi_0 = b, psi_-1 = c e^{-2 pi i 2 x/L} with |a b| > |b c|:
    F_perp = sqrt2 (conj(a) b e^{-2 pi i 3 x/L} + conj(b) c e^{-2 pi i 2 x/L}) is dominated by
    its first term, so it winds -3 times (argument principle)."""
    n = 512
    x = np.arange(n)
    field = np.stack([0.5 * np.exp(2j * np.pi * 3 * x / n), 0.8 + 0 * x, 0.2 * np.exp(-2j * np.pi * 2 * x / n)])
    b = B.GPEBatch((n,), 2, "c128")
    b.set_mean_field(torch.as_tensor(field))
    b.init_noise(1, (0.0,) * 6, 0.0)
    nb, sd = b.layout()
    acc = b.new_accumulator(1)
    b.observables(acc, B.GPE_OBS_WINDING, 0)
    np.testing.assert_allclose(B.unpack_winding(acc, nb, 2), [-3.0, -3.0], atol=1e-12)
    b.close()


def test_winding_needs_1d(B):
    b = B.GPEBatch((64, 64), 1, "c128")
    acc = b.new_accumulator(1)
    with pytest.raises(B.GPEError) as ei:
        b.observables(acc, B.GPE_OBS_WINDING, 0)
    assert ei.value.status == B.GPE_EUNSUPPORTED
    b.close()


def test_coarsening_driver_small(B):
    from paper_2310_03636_gb300 import coarsening1d
    res, arr = coarsening1d.run(n=1024, ntraj=8, dt=0.04, t_end=400.0, nsamples=6, t_first=40.0, t_fit=100.0,
                                kmax_ir=0.3)
    assert res["steps"] == 10000
    assert res["norm_drift"] < 2e-5
    assert res["winding_integer_dev"] < 1e-6
    assert arr["S_perp"].shape == (len(arr["times"]), 513)
    # the spin instability of the polar state (unstable band k^2/2 < 2 n |c1| - q) lifts
    # S_perp far above its initial noise level there
    kq = (arr["k"] > 0.05) & (arr["k"] < 0.4)
    assert arr["S_perp"][-1][kq].mean() > 10 * arr["S_perp"][0][kq].mean()
    for key in ("beta_moment", "beta_collapse"):
        assert np.isfinite(res[key])


def test_sweep3d_driver_against_oracle(B):
    """The 3D quench-sweep driver (sweep3d.run_one) in FP64 on a small grid: its per-sample
    totals and drifts of N, F_z and E equal those of the oracle's run of the same steps
    (diagnostics of the oracle's fields at the same sample times, the same summary)."""
    from oracle.philox import tw_noise
    from paper_2310_03636_gb300 import sweep3d
    n, ntraj, steps, every, q, dt, seed = 64, 1, 40, 20, 0.15, 0.02, 20231005
    r = sweep3d.run_one(n, ntraj, q, steps, every, dt=dt, seed=seed, dtype="c128")
    psi = np.stack([tw_noise((n, n, n), seed, t, 0.5, 1.0) for t in range(ntraj)])
    psi[:, 1] += 1.0
    p = torch.as_tensor(psi)
    recs = [O.diagnostics(p, 1.0, 1.0, -0.1, q, 3).numpy()]
    for _ in range(steps // every):
        p = O.propagate(p, dt, every, 1.0, -0.1, q, 1.0, 3)
        recs.append(O.diagnostics(p, 1.0, 1.0, -0.1, q, 3).numpy())
    ref = sweep3d.drift_summary(np.stack(recs))
    for key in ("N", "F_z", "E"):
        np.testing.assert_allclose(r[key], ref[key], rtol=1e-10, atol=1e-9 * abs(ref["N"][0]), err_msg=key)
    for key in ("max_rel_dN", "max_rel_dFz", "max_rel_dE"):
        np.testing.assert_allclose(r[key], ref[key], rtol=1e-3, atol=1e-12, err_msg=key)
    assert max(r["max_rel_dN"]) < 1e-12
