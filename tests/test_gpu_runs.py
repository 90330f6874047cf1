"""GPU parity of the row-OR contraction on operands whose set bits come in runs
(the thick curves a plot gives): runs from single bits to whole rows cover
every block level of the tables (1, 4, 16 and 64 rows of B), alternating bits
overflow one list window, ragged K masks the last word, and a K too long for
one tile is split into chunks OR-ed together.  Every bit equals the oracle's."""
import numpy as np
import pytest

import paper_1609_00061_gb300 as pa

from test_gpu_parity import check_same, pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = pa.Engine(0)
    e.set_path("rowor")
    yield e
    e.close()


def run_rows(rng, M, K):
    """Rows of A: empty, all ones, one run of random length at a random place,
    several runs, alternating bits, sparse random bits."""
    A = np.zeros((M, K), dtype=np.uint8)
    for i in range(M):
        kind = i % 6
        if kind == 1:
            A[i, :] = 1
        elif kind == 2:
            L = int(rng.integers(1, min(K, 200) + 1))
            s = int(rng.integers(0, K - L + 1))
            A[i, s:s + L] = 1
        elif kind == 3:
            for _ in range(int(rng.integers(1, 6))):
                L = int(rng.integers(1, min(K, 90) + 1))
                s = int(rng.integers(0, K - L + 1))
                A[i, s:s + L] = 1
        elif kind == 4:
            A[i, int(rng.integers(0, 2))::2] = 1
        elif kind == 5:
            A[i] = rng.random(K) < 0.05
    return A


@pytest.mark.parametrize("M,K,N", [(60, 63, 130), (60, 64, 64), (72, 65, 200), (90, 1000, 100),
                                   (48, 2048, 2048), (30, 10000, 128)])
def test_runs(eng, orc, M, K, N):
    rng = np.random.default_rng(5000 + K)
    A = run_rows(rng, M, K)
    B = (rng.random((K, N)) < 0.03).astype(np.uint8)
    want = orc.contract(orc.Arr(A, (0, 1)), orc.Arr(B, (1, 2)), (0, 2), [M, K, N]).data
    got = eng.contract(pack(A, (0, 1)), pack(B, (1, 2)), (0, 2))
    eng.sync()
    check_same(got, want, f"M={M} K={K} N={N}")


def test_runs_banded_b(eng, orc):
    """B with runs too (a band per row), so that block ORs of B differ from
    their single rows in structured ways."""
    rng = np.random.default_rng(77)
    M, K, N = 64, 700, 900
    A = run_rows(rng, M, K)
    B = np.zeros((K, N), dtype=np.uint8)
    for k in range(K):
        c = int((N - 40) * (0.5 + 0.5 * np.sin(k / 50.0)))
        B[k, c:c + int(rng.integers(1, 40))] = 1
    want = orc.contract(orc.Arr(A, (0, 1)), orc.Arr(B, (1, 2)), (0, 2), [M, K, N]).data
    got = eng.contract(pack(A, (0, 1)), pack(B, (1, 2)), (0, 2))
    eng.sync()
    check_same(got, want)

