"""The test helper that refits the oracle on a given dictionary: on the
oracle's own final dictionaries it must give the oracle's own coefficients
and surrogate (the Elastic Net minimiser of Eq. (2) is unique)."""
import numpy as np

import oracle
from oracle_refit import model_with, oracle_on_gpu_dictionary, refit_on_dictionary
from paper_2605_16564_gb300 import fields


def test_refit_on_the_oracles_own_dictionary_reproduces_its_fit():
    K = fields.voronoi_field(64, n_sites=9, seed=51)
    params = oracle.default_params(k_top=6, levels=2)
    ref = oracle.fit_all(K, (64, 64), (2, 2), 2, (4, 4), params)
    pts = fields.cell_centred_points((64, 64), (1.0, 1.0))
    ko, own = oracle.evaluate(ref, pts, return_owner=True)
    for s in range(4):
        m = int(ref["M"][s])
        b = refit_on_dictionary((64, 64), ref["boxes"][s], ref["c"][s, :m], K)
        assert np.abs(b - ref["beta"][s, :m]).max() <= 1e-10 * max(1.0, np.abs(ref["beta"][s, :m]).max())
        q = own == s
        kr = oracle_on_gpu_dictionary((64, 64), ref, ref, s, K, pts[q])
        np.testing.assert_allclose(kr, ko[q], rtol=1e-10, atol=0)


def test_model_with_replaces_one_subdomain_only():
    K = fields.voronoi_field(32, n_sites=5, seed=52)
    ref = oracle.fit_all(K, (32, 32), (2, 1), 1, (3, 3), oracle.default_params(k_top=2, levels=1))
    c = ref["c"][0, :4].copy()
    mdl = model_with(ref, 0, c, np.full(4, np.log(3.0)))
    pts = fields.cell_centred_points((32, 32), (1.0, 1.0))
    k_new, own = oracle.evaluate(mdl, pts, return_owner=True)
    k_ref = oracle.evaluate(ref, pts)
    np.testing.assert_allclose(k_new[own == 0], 3.0, rtol=1e-13)  # constant coefficients: K* = 3
    np.testing.assert_array_equal(k_new[own == 1], k_ref[own == 1])
