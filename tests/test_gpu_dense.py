"""The landmark-space FP64 product engines against numpy FP64."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1705_10887_gb300 as sb  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sb.build()
    sb.library()


def _check(A, B, C, slack=1.0):
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    K = A.shape[1]
    err = np.abs(C - ref)
    # slicing keeps 48 bits per row of A and column of B; FP64 sums add K ulps
    assert np.all(err <= slack * (K * 2.0 ** -46) * bound + 1e-300), (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("M, N, K", [(300, 200, 1000), (128, 64, 64), (1, 1, 1), (700, 33, 5000)])
def test_tc_matches_fp64(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(K, N))
    C = sb.dgemm(A, B, sb.DENSE_TC)
    _check(A, B, C)
    C64 = sb.dgemm(A, B, sb.DENSE_FP64)
    _check(A, B, C64)


def test_tc_scales_and_zero_rows():
    rng = np.random.default_rng(7)
    M, N, K = 257, 130, 777
    A = rng.normal(size=(M, K)) * (10.0 ** rng.uniform(-150, 150, size=(M, 1)))
    B = rng.normal(size=(K, N)) * (10.0 ** rng.uniform(-150, 150, size=(1, N)))
    A[5] = 0.0
    B[:, 7] = 0.0
    C = sb.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), sb.DENSE_TC).cpu().numpy()
    assert np.all(C[5] == 0.0) and np.all(C[:, 7] == 0.0)
    _check(A, B, C)


def test_tc_nonnegative_harmonic_like():
    # entries in [0, 1] with a few near 1, like harmonic measures; products are accurate to 2^-46 of |A||B|
    rng = np.random.default_rng(11)
    M, N, K = 400, 400, 20000
    A = rng.random((M, K)) ** 8
    B = A.T.copy() * rng.random((K, 1))
    C = sb.dgemm(A, B, sb.DENSE_TC)
    _check(A, B, C)


def test_dgemm_rejects_bad_mode():
    with pytest.raises(sb.SbhaError):
        sb.dgemm(np.ones((2, 2)), np.ones((2, 2)), 9)
