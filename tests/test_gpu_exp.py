"""The table-driven exponential of the rate kernels (Tang, ACM TOMS 15, 1989) against CUDA's
exp (through torch) and glibc's exp, over the argument range the rates use."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_12070_gb300 import chem

pytestmark = pytest.mark.gpu


def test_exp_matches_library_exp():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-707.0, 707.0, 200000), rng.uniform(-1.0, 1.0, 50000),
                        np.array([0.0, -0.0, 1e-300, -1e-300, 0.5, -0.5, 700.0, -700.0, 707.9, -707.9]),
                        np.log(2.0) / 64 * np.arange(-64, 65)])
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    chem.chem_debug_exp(xd, y)
    ref_gpu = torch.exp(xd)
    torch.cuda.synchronize()
    y, ref_gpu = y.cpu().numpy(), ref_gpu.cpu().numpy()
    ref_cpu = np.exp(x)
    rel_gpu = np.abs(y - ref_gpu) / np.abs(ref_gpu)
    rel_cpu = np.abs(y - ref_cpu) / np.abs(ref_cpu)
    eps = np.finfo(np.float64).eps
    assert rel_gpu.max() <= 2 * eps, rel_gpu.max()
    assert rel_cpu.max() <= 2 * eps, rel_cpu.max()
    # most results are correctly rounded
    assert np.mean(y == ref_cpu) > 0.95


def test_exp_edges_fall_back():
    x = np.array([708.5, -708.5, 709.7, -745.0, -800.0, 800.0, np.inf, -np.inf, np.nan])
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    chem.chem_debug_exp(xd, y)
    ref = torch.exp(xd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), ref.cpu().numpy())
