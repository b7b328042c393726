import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def workload_rows(wl, q=0, k_range=None):
    """Full Z as rows (N, K), per-column Delta and the omega grid for a (small) workload, from the generators."""
    from synthetic import workloads as W
    import oracle

    n_pb = wl.n_pb(q)
    ks = range(wl.n_k) if k_range is None else k_range
    zs, ds = [], []
    for k in ks:
        nu = wl.n_unocc(q, k)
        zt = W.z_block(wl.seed, q, k, n_pb, wl.n_occ, nu, wl.s_div)
        zs.append(zt.T)
        d, bad = oracle.delta(W.eps_occ(wl.seed, q, k, wl.n_occ), W.eps_unocc(wl.seed, q, k, nu))
        assert bad == 0
        ds.append(d)
    return np.ascontiguousarray(np.concatenate(zs, axis=1)), np.concatenate(ds), wl.omega


@pytest.fixture(scope="session")
def tiny_oracle():
    """Oracle chi0, eps, W for the tiny workload (n_pb=64, K=2048, 6 frequencies)."""
    from synthetic import TINY, coulomb_v
    import oracle

    Z, d, om = workload_rows(TINY)
    chi = oracle.chi0_full(Z, d, om, TINY.spin)
    v = coulomb_v(TINY.seed, 0, TINY.n_pb(0))
    eps, W, Wc, info = oracle.eps_w(chi, v)
    return dict(Z=Z, delta=d, omega=om, chi=chi, v=v, eps=eps, W=W, Wc=Wc, info=info, spin=TINY.spin)
