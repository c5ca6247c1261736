"""Test helper: the oracle's Elastic Net fit on a dictionary the GPU chose.

Where fp32 rounding moves a marking decision of the mixed form, its refined
dictionary differs from the oracle's and the two surrogates are not
comparable cell by cell. The per-cell bar is then checked against the
oracle's own fit (assembly, Gram and Elastic Net of Eq. (2), section 3) of
the GPU's final dictionary of that subdomain, so that every sampled
subdomain meets the per-cell bar and not only those whose dictionaries
agree. Oracle calls only; nothing here comes from the CUDA path but the
dictionary being refitted.
"""
import numpy as np

import oracle


def refit_on_dictionary(n_cells, box, c, K, lambda1_hat=4.59e-4, lambda2_hat=4.64e-6):
    """Coefficients of the oracle's fit of the patch box[6:12] with centres c [M, 4]."""
    dim = len(n_cells)
    x, y, _ = oracle.box_cells(n_cells, box[6:9], box[9:12], K)
    W = oracle.assemble(dim, x, c)
    G, b = oracle.gram(W, y)
    N = x.shape[0]
    beta, info = oracle.enet(G, b, N * lambda1_hat, N * lambda2_hat)
    assert info["certified"]
    return beta


def model_with(ref, s, c, beta):
    """A copy of the oracle model `ref` with subdomain s's dictionary and
    coefficients replaced (capacity grown if needed)."""
    M = c.shape[0]
    mc = max(int(ref["m_cap"]), M)
    out = dict(ref)
    cc = np.zeros((ref["c"].shape[0], mc, 4))
    cc[:, :ref["c"].shape[1]] = ref["c"]
    bb = np.zeros((ref["beta"].shape[0], mc))
    bb[:, :ref["beta"].shape[1]] = ref["beta"]
    cc[s, :M] = c
    cc[s, M:] = 0.0
    bb[s, :M] = beta
    bb[s, M:] = 0.0
    MM = np.array(ref["M"]).copy()
    MM[s] = M
    out.update(c=cc, beta=bb, M=MM, m_cap=mc)
    return out


def oracle_on_gpu_dictionary(n_cells, ref, got, s, K, pts, **lam):
    """The oracle's K* at pts (owned by s) from its fit of the GPU's dictionary of s."""
    m = int(got["M"][s])
    c = np.array(got["c"][s, :m])
    beta = refit_on_dictionary(n_cells, ref["boxes"][s], c, K, **lam)
    return oracle.evaluate(model_with(ref, s, c, beta), pts)
