"""Host side of topk_frequent (CPU only): the sampling rate and k* the
library plans from eps and delta equal the oracle's, and bad arguments are
refused before any device work."""
import ctypes

import pytest

import oracle


@pytest.fixture(scope="module")
def tk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03942_gb300 as tk
    return tk


@pytest.mark.parametrize("n", [1000, 1 << 26, 1 << 28, 1 << 40])
@pytest.mark.parametrize("eps,delta", [(3e-4, 1e-4), (1e-6, 1e-8), (1e-2, 1e-3)])
@pytest.mark.parametrize("pes", [1, 64, 2048])
def test_plan_matches_oracle(tk, n, eps, delta, pes):
    for alg in (tk.TOPK_FREQ_PAC, tk.TOPK_FREQ_EC):
        fp = tk.make_freq_params(32, algorithm=alg, epsilon=eps, delta=delta, pes=pes)
        rho, kstar = tk.topk_frequent_plan(n, fp)
        want = oracle.frequent_plan(n, 32, eps, delta, pes=pes, exact=alg == tk.TOPK_FREQ_EC)
        assert kstar == want[1]
        assert rho == pytest.approx(want[0], rel=1e-14)


def test_plan_and_call_reject_bad_arguments(tk):
    lib = tk.load_library()
    rho, ks = ctypes.c_double(), ctypes.c_uint32()
    bad = [tk.make_freq_params(0), tk.make_freq_params(4, algorithm=7), tk.make_freq_params(4, epsilon=0.0),
           tk.make_freq_params(4, delta=1.0), tk.make_freq_params(4, rho=1.5), tk.make_freq_params(4, kstar=3)]
    for fp in bad:
        assert lib.topk_frequent_plan(1000, ctypes.byref(fp), ctypes.byref(rho), ctypes.byref(ks)) == tk.TOPK_EINVAL
    assert lib.topk_frequent_plan(0, ctypes.byref(tk.make_freq_params(4)), ctypes.byref(rho),
                                  ctypes.byref(ks)) == tk.TOPK_EINVAL
    fp = tk.make_freq_params(4)
    assert lib.topk_frequent(None, None, 10, tk.TOPK_U32, ctypes.byref(fp), None, None, None, None) == tk.TOPK_EINVAL
