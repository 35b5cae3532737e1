"""The findings Sec. 5.2 states about Fig. 1 a-e, checked on a reduced sweep
(6 realisations of the SBM N = 1e3, k = 20, s = 16 at eps = 0.02 and 0.04)
through csc_cluster, with spectral clustering (Alg. 1, oracle) on the same graphs.
The full sweep is tests/fig1_sweep.py."""
import pytest

from . import fig1_sweep as fs

pytestmark = pytest.mark.gpu

csc = pytest.importorskip("paper_1602_02018_gb300")


@pytest.fixture(scope="module")
def sweep():
    from paper_1602_02018_gb300 import build

    build.build()
    return fs.run({"a", "c", "d", "e"}, 6, eps_grid=[0.02, 0.04], workers=6)["hom"]


def test_lambda_k_estimate_lies_between_lambda_k_and_lambda_k1(sweep):
    """Fig. 1 e: the estimate overshoots lambda_k but stays below lambda_(k+1) for small eps."""
    for e in (0.02, 0.04):
        assert sweep[e]["est_in_gap"] == 1.0
        assert sweep[e]["lam_est"] > sweep[e]["lk"]


def test_recovery_saturates_at_the_default_n(sweep):
    """Fig. 1 a: doubling n past 2 k ln k changes little; n = k is far worse."""
    n_vals = fs.variants()["a"][1]
    r = sweep[0.02]["csc"]
    assert r[("a", n_vals[3])] - r[("a", n_vals[2])] <= 0.03
    assert r[("a", n_vals[0])] < r[("a", n_vals[2])] - 0.1


def test_recovery_saturates_at_the_default_degree_and_gamma(sweep):
    """Fig. 1 c-d: m = 100 and gamma = 0.1 add nothing over m = 50 and gamma = 1e-3."""
    for e in (0.02, 0.04):
        r = sweep[e]["csc"]
        assert abs(r[("c", 100)] - r[("c", 50)]) <= 0.03
        assert abs(r[("d", 0.1)] - r[("d", 1e-3)]) <= 0.03


def test_csc_close_to_spectral_clustering(sweep):
    """Sec. 5.2: CSC recovers the communities nearly as well as SC for small eps."""
    assert sweep[0.02]["csc"][("def", None)] >= sweep[0.02]["sc"] - 0.05
    assert sweep[0.04]["csc"][("def", None)] >= sweep[0.04]["sc"] - 0.1


def test_highpass_regulariser_not_worse(sweep):
    """The discussion after Eq. 5 prefers g = 1 - h~; it is at least as good as L^4 here."""
    for e in (0.02, 0.04):
        assert sweep[e]["csc"][("hp", None)] >= sweep[e]["csc"][("def", None)] - 0.02
