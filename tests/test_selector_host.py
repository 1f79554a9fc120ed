"""Host-side pieces of the selector module, on the CPU: labels from measured orthogonalities and the
network's initial parameters.  (The selector's orchestration runs in the C library and is tested on the GPU.)"""
import numpy as np

from oracle import mlp
from paper_1401_5171_gb300 import selector


def test_labels_are_the_cheapest_option_meeting_tol():
    inf = np.inf
    orth = np.array([[1e-13, 1e-15, 1e-15],      # one pass suffices
                     [3e-12, 2e-15, 1e-15],      # two passes
                     [inf, inf, 4e-15],          # only the shifted option completes
                     [inf, inf, inf],            # nothing completes: the most robust option
                     [2e-11, 5e-12, 3e-12]])     # nothing meets tol: the most robust option
    assert selector.labels_from(orth, 1e-12).tolist() == [0, 1, 2, 2, 2]
    assert selector.labels_from(orth, 1e-11).tolist() == [0, 0, 2, 2, 1]


def test_initial_parameters_layout():
    p = selector.init_params(1)
    assert p.dtype == np.float32 and p.size == mlp.COUNT
    assert np.array_equal(p, selector.init_params(1))
