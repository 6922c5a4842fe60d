"""Well-prepared initial data on the GPU (sgn_well_prepare, Sec. 3.2) against
the oracle's plain definition (oracle/well_prepared.py): FP64 within 1e-12 per
field, mixed precision within 1e-5, rows with a dry cell unchanged, and the
App. B solitary wave's w and p reproduced to discretisation accuracy."""
import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_12162_gb300 import build, sgn
    build.build()
    sgn.load()
    return sgn


def _rows_case(nx=300, ny=6, dx=0.1, seed=3):
    """Smooth data varying along x, different in every row; the last row has a
    dry cell."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) * dx
    b = np.empty((ny, nx))
    q = np.zeros((5, ny, nx))
    for j in range(ny):
        k = rng.uniform(0.3, 1.0, 3)
        b[j] = -1.0 + 0.3 * np.sin(k[0] * x) * np.exp(-((x - 15.0) / 8.0) ** 2)
        h = -b[j] + 0.1 * np.exp(-((x - rng.uniform(10, 20)) / 2.0) ** 2)
        q[0, j] = b[j] + h
        q[1, j] = h * 0.3 * np.cos(k[1] * x)
    i = nx // 3
    b[-1, i] = 0.5                        # a dry cell: the row stays as it is
    q[0, -1, i] = 0.5
    q[1, -1, i] = 0.0
    return b, q, dx


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_well_prepared_matches_oracle(S, oracle_mod, precision, tol):
    from oracle import well_prepared as WP
    b, q, dx = _rows_case()
    s = S.Solver(b, model=1, dx=dx, bc=(1, 1, 1, 1), h_star=0.0, precision=precision)
    s.set_state(q)
    before = s.get_state()[0]
    s.well_prepare()
    after = s.get_state()[0]
    ref = WP.well_prepared(before, b, dx)
    for k in (3, 4):
        for j in range(b.shape[0]):
            den = np.linalg.norm(ref[k, j])
            err = np.linalg.norm(after[k, j] - ref[k, j]) / (den if den > 0 else 1.0)
            assert err <= tol, (k, j, err)
    assert np.array_equal(after[:3], before[:3])
    assert np.array_equal(after[3:, -1], before[3:, -1])      # the row with a dry cell
    assert s.next_dt() > 0.0


def test_well_prepared_solitary_wave(S):
    N, L = 800, 40.0
    dx = L / N
    x = (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(x, np.arange(4) * dx)
    b = -np.ones_like(X)
    q = W.soliton_state(1, X, Y, b, 0.2, 1.0, 20.0)
    ill = q.copy()
    ill[3:] = 0.0
    s = S.Solver(b, model=1, dx=dx, bc=(1, 1, 0, 0), h_star=0.0)
    s.set_state(ill)
    s.well_prepare()
    out = s.get_state()[0]
    for k in (3, 4):
        assert np.abs(out[k] - q[k]).max() <= 2e-3 * np.abs(q[k]).max()


def test_well_prepare_rejects_other_models(S):
    b, q, dx = _rows_case(nx=20, ny=2)
    s = S.Solver(b, model=2, dx=dx)
    with pytest.raises(S.SGNError):
        s.well_prepare()
