"""Parity of the library's Kmouflage background solver (mg_kmo_background,
host code behind the C ABI) with the FP64 oracle of oracle/background.py,
and its argument handling.  Both integrate to a local tolerance of 1e-12;
the tables agree to 1e-9 relative."""
import numpy as np
import pytest

from oracle import background as ob

pytestmark = pytest.mark.gpu

from test_gpu_parity import B  # noqa: E402,F401

A_OUT = np.array([1e-5, 3e-4, 2e-3, 0.02, 0.1, 0.25, 0.5, 0.75, 1.0, 1.3])


@pytest.mark.parametrize("n,k0,beta", [(2, 1.0, 0.2), (2, 10.0, 0.2), (3, 1.0, 0.2), (2, 100.0, 0.3),
                                       (2, 0.0, 0.1)])
def test_background_matches_oracle(B, n, k0, beta):
    rc, lam, tab = B.mg_kmo_background(B.kmo_background_params(n=n, k0=k0, beta_kmo=beta), A_OUT)
    lam_o, ref = ob.solve(ob.Background(n=n, k0=k0, beta=beta), A_OUT)
    assert rc == 0
    assert lam == pytest.approx(lam_o, rel=1e-11)
    np.testing.assert_allclose(tab[:, 0], ref[:, 0], rtol=1e-11)          # H/H0
    np.testing.assert_allclose(tab[:, 3], ref[:, 3], rtol=1e-11)          # A
    for c in (1, 2, 4):                                                    # phibar, dphibar/da, phibar'/H0
        big = np.abs(ref[:, c]) > 1e-20
        np.testing.assert_allclose(tab[big, c], ref[big, c], rtol=1e-9)
    assert tab[-2, 0] == pytest.approx(1.0, abs=1e-12)                    # H(a=1) = H0


def test_uncoupled_background_is_lcdm(B):
    p = B.kmo_background_params(beta_kmo=0.0)
    rc, lam, tab = B.mg_kmo_background(p, A_OUT)
    bg = ob.Background(beta=0.0)
    om, orad = bg.omega_m, bg.omega_r
    assert lam ** 2 == pytest.approx(3.0 * (1.0 - om - orad), rel=1e-11)
    np.testing.assert_allclose(tab[:, 0], np.sqrt(orad / A_OUT ** 4 + om / A_OUT ** 3 + 1.0 - om - orad),
                               rtol=1e-11)
    assert np.abs(tab[:, 1]).max() < 1e-20


def test_given_lambda_and_any_order(B):
    p = B.kmo_background_params(k0=10.0)
    _, lam, tab = B.mg_kmo_background(p, A_OUT)
    perm = np.random.default_rng(3).permutation(A_OUT.size)
    rc, lam2, tab2 = B.mg_kmo_background(p, A_OUT[perm], lam=lam)
    assert rc == 0 and lam2 == lam
    np.testing.assert_allclose(tab2, tab[perm], rtol=1e-10, atol=1e-300)
    _, ref = ob.solve(ob.Background(k0=10.0), A_OUT, lam=lam)
    np.testing.assert_allclose(tab[:, 0], ref[:, 0], rtol=1e-11)


def test_background_arguments(B):
    good = dict(n=2, k0=1.0)
    for bad in (dict(n=1), dict(k0=-1.0), dict(omega_m=1.0), dict(a_ini=0.0), dict(rtol=1e-20),
                dict(h0_tol=0.0), dict(h=-0.7)):
        p = B.kmo_background_params(**{**good, **bad})
        with pytest.raises(B.MGError) as e:
            B.mg_kmo_background(p, A_OUT)
        assert e.value.code == B.MG_ERR_ARG
    p = B.kmo_background_params(**good)
    for a in ([1e-6], [200.0], [np.nan]):
        with pytest.raises(B.MGError):
            B.mg_kmo_background(p, a)
    # an unreachable shooting tolerance is a warning with the last lambda's table
    rc, lam, tab = B.mg_kmo_background(B.kmo_background_params(h0_tol=1e-300), [1.0])
    assert rc == B.MG_WARN_NOT_CONVERGED and tab[0, 0] == pytest.approx(1.0, abs=1e-12)
