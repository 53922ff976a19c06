"""The all-core CPU baseline (oracle/stencil_omp.c: Jacobi split over planes, Gauss-Seidel
pipeline-parallel over row blocks as in the paper's Sec. 3) gives the serial oracle's bits for any
thread count, ragged grids, f, several sweeps."""
import numpy as np
import pytest

import oracle
from paper_1004_1741_gb300 import workloads as W


@pytest.mark.parametrize("dims", [(13, 11, 9), (1, 1, 1), (5, 1, 7), (20, 3, 2), (31, 40, 6)])
@pytest.mark.parametrize("threads", [1, 2, 3, 4, 7])
def test_omp_baseline_matches_the_oracle(dims, threads):
    u0, f0 = W.random_grid(*dims, seed=sum(dims) + threads, with_f=True)
    for f, ns in ((None, 1), (f0, 5)):
        np.testing.assert_array_equal(oracle.gs_lex_omp(u0, f, 0.1, ns, threads=threads),
                                      oracle.gs_lex(u0, f, 0.1, ns))
        np.testing.assert_array_equal(oracle.jacobi_omp(u0, f, 0.1, ns, threads=threads),
                                      oracle.jacobi(u0, f, 0.1, ns))
    np.testing.assert_array_equal(oracle.jacobi_omp(u0, f0, 0.1, 3, a=1 / 7, b=1 / 7, threads=threads),
                                  oracle.jacobi(u0, f0, 0.1, 3, a=1 / 7, b=1 / 7))


def test_omp_gs_pipeline_many_planes_and_sweeps():
    """More row blocks than fit evenly, many planes and sweeps: the cross-block waits keep the serial order."""
    u0, f0 = W.random_grid(23, 64, 37, seed=3, with_f=True)
    np.testing.assert_array_equal(oracle.gs_lex_omp(u0, f0, 0.05, 7, threads=9), oracle.gs_lex(u0, f0, 0.05, 7))


def test_omp_baseline_uses_threads():
    assert oracle.omp_threads() >= 1
