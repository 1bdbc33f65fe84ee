"""Host-side summary of the 3D quench sweep's diagnostics records (no GPU)."""
import numpy as np

from paper_2310_03636_gb300.sweep3d import drift_summary


def test_drift_summary_totals_and_drifts():
    # two samples x two trajectories of (N_1, N_0, N_-1, E_kin, E_q, E_c0, E_c1, E_V)
    d = np.zeros((2, 2, 8))
    d[0, 0] = [1.0, 2.0, 1.0, 0.5, 0.2, 3.0, -0.1, 0.0]      # N 4, F_z 0, E 3.6
    d[0, 1] = [0.5, 3.0, 0.5, 0.4, 0.1, 4.0, -0.2, 0.0]      # N 4, F_z 0, E 4.3
    d[1, 0] = [1.1, 1.9, 1.0, 0.6, 0.2, 3.0, -0.1, 0.0]      # N 4, F_z 0.1, E 3.7
    d[1, 1] = [0.5, 3.0, 0.5, 0.4, 0.1, 4.0, -0.2, 0.43]     # N 4, F_z 0, E 4.73
    s = drift_summary(d)
    np.testing.assert_allclose(s["N"], [8.0, 8.0])
    np.testing.assert_allclose(s["F_z"], [0.0, 0.1])
    np.testing.assert_allclose(s["E"], [7.9, 8.43])
    np.testing.assert_allclose(s["max_rel_dN"], [0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(s["max_rel_dFz"], [0.0, 0.1 / 4.0])
    np.testing.assert_allclose(s["max_rel_dE"], [0.0, max(0.1 / 3.6, 0.43 / 4.3)])
