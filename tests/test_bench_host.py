"""Host-side arithmetic of bench.py's energy report (CPU, no GPU): the
speedup bound it evaluates is the oracle's Eq. (speedup), and its one-GPU
cost model reduces to the exact work ratio in the cases that fix it."""
import pytest

import bench
from oracle import modal


@pytest.mark.parametrize("n_p", [4, 8, 32, 128])
@pytest.mark.parametrize("k", [1, 3, 12])
@pytest.mark.parametrize("ratio", [0.05, 0.4, 1.7])
def test_speedup_bound_is_the_oracle_model(n_p, k, ratio):
    assert bench.s_bound(n_p, k, 1 / 16, ratio) == pytest.approx(modal.s_bound(n_p, k, 1 / 16, ratio),
                                                                 rel=1e-15)


def test_one_gpu_cost_model_closed_forms():
    # one iteration over all slices with no coarse cost and the batched step
    # as fast as the serial one: exactly the serial fine work
    g = bench.gamma_terms(32, 1, 256, 8, 1e-5, 1e-5, 0.0, 2.0, 1.0)
    assert g["gamma_bound_one_gpu"] == pytest.approx(1.0, rel=1e-15)
    assert g["t_ratio_measured"] == 2.0
    # K iterations: sum_{j<K} (N - j) slice-sweeps of N_f steps over N N_f
    n_p, k = 32, 12
    g = bench.gamma_terms(n_p, k, 256, 8, 1e-5, 1e-5, 0.0, 1.0, 1.0)
    assert g["gamma_bound_one_gpu"] == pytest.approx(sum(n_p - j for j in range(k)) / n_p, rel=1e-14)
    # the coarse chain alone: the start-up chain (N G's) plus N - j - 1 per iteration
    g = bench.gamma_terms(n_p, k, 256, 8, 1e-5, 0.0, 2e-6, 1.0, 1.0)
    coarse = (n_p + sum(n_p - j - 1 for j in range(k))) * 8 * 2e-6
    assert g["gamma_bound_one_gpu"] == pytest.approx(coarse / (n_p * 256 * 1e-5), rel=1e-14)
    # the paper's bound: N_p / S_bound
    assert g["gamma_bound_paper"] == pytest.approx(n_p / modal.s_bound(n_p, k, 8 / 256, 0.2), rel=1e-14)
