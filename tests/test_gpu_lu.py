"""The kernels' dense LU with partial pivoting (Sec. 2.3: dense LU + back substitution), through
chem_debug_lu: its schedule with two barriers per column (the integrate kernels' default) and its
panel-blocked schedule give bitwise the factors of the column-by-column one in every factor
precision (the same pivots and the same operations on every entry, in the same order), and the FP64 factors equal LAPACK's (scipy.linalg.lu_factor, whose pivot is also the
first largest |a|) on random matrices, with reciprocal pivots within one unit in the last place.
The factors are stored as P A = L D U' (U' = D^-1 U, unit upper): the upper factor is rebuilt
from them as U = D U' for the comparison.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2105_12070_gb300 import chem  # noqa: E402

PRECISIONS = (chem.CHEM_PREC_FP64, chem.CHEM_PREC_MIXED, chem.CHEM_PREC_MIXED_FF)


def _matrices(N, n, seed):
    """Random matrices, iteration-matrix-like ones (a large diagonal over a stiff spread of scales)
    and columns with tied |a| (ties must go to the lowest row)."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, N, N))
    for m in range(n // 3, 2 * n // 3):
        scale = 10.0 ** rng.uniform(-8, 8, size=N)
        A[m] = rng.normal(size=(N, N)) * scale[None, :]
        A[m][np.diag_indices(N)] += 10.0 ** rng.uniform(0, 12)
    for m in range(2 * n // 3, n):
        k = rng.integers(0, N)
        A[m][:, k] = np.sign(rng.normal(size=N)) * 2.0  # every |a| in column k equal
    return A


@pytest.mark.parametrize("N", [1, 2, 5, 8, 9, 16, 31, 32, 33, 53, 64, 65, 100, 128])
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("variant", [1, 2])
def test_lu_schedules_bitwise_equal(N, prec, variant):
    A = torch.from_numpy(_matrices(N, 24, 1000 + N)).cuda()
    ref = chem.chem_debug_lu(A, prec, variant=0)
    out = chem.chem_debug_lu(A, prec, variant=variant)
    torch.cuda.synchronize()
    for r, o in zip(ref, out):
        assert torch.equal(r.view(torch.int32), o.view(torch.int32)), (N, prec, variant)


@pytest.mark.parametrize("N", [5, 53, 100])
def test_fp64_lu_matches_lapack(N):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    A = _matrices(N, 12, 2000 + N)[: 2 * 12 // 3]  # no tied columns: pivots are unique
    F, D, P, S = (t.cpu().numpy() for t in chem.chem_debug_lu(torch.from_numpy(A).cuda(), chem.CHEM_PREC_FP64,
                                                               variant=1))
    for m in range(A.shape[0]):
        lu, piv = scipy_linalg.lu_factor(A[m])
        perm = np.arange(N)
        for k, p in enumerate(piv):
            perm[[k, p]] = perm[[p, k]]
        np.testing.assert_array_equal(P[m], perm)
        f = F[m].reshape(N, N).copy()
        # U = D U': the strictly upper part row by row times the pivot on the diagonal
        up = np.triu(np.ones((N, N), dtype=bool), 1)
        f[up] = (f * np.diag(f)[:, None])[up]
        scale = np.abs(lu).max(axis=1, keepdims=True)
        assert np.all(np.abs(f - lu) <= 1e-10 * scale), m
        # the reciprocal pivots (Newton's iteration): within one unit in the last place of 1 / u_kk
        d_exact = 1.0 / np.diag(f)
        assert np.all(np.abs(D[m] - d_exact) <= np.spacing(np.abs(d_exact))), m
        assert S[m] == 0


def test_singular_flag():
    N = 20
    A = np.random.default_rng(3).normal(size=(2, N, N))
    A[1][:, 7] = 0.0  # an exactly zero column
    for variant in (0, 1, 2):
        *_, S = chem.chem_debug_lu(torch.from_numpy(A).cuda(), chem.CHEM_PREC_FP64, variant=variant)
        assert S.cpu().tolist() == [0, 1]
