"""Full-size parity of the off-surface double layer (Sections 2 and 3.2): the starfish
boundary (N_Gamma = 6144, 6 curves x 1024 nodes) at sampled targets in all three
near-boundary regimes, binary64, against the oracle's rules.  The 0.1 h_s targets sit on
node normals, so their foot points coincide with boundary nodes: the case where the
normal-line rule's trigonometric interpolation weights are most prone to cancellation."""
import numpy as np
import pytest

import mh_workloads as W
from oracle import bie, geometry as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import paper_1007_5335_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(mh):
    return mh.Context(0)


def test_full_size_starfish_off_surface_sampled(mh, ctx):
    """N_Gamma = 6144 (6 curves x 1024): U^h at 40 random points of the unit disk that fall in
    Omega and at points 3, 0.5 and 0.1 h_s from two nodes of every curve (the upsampled and the
    normal-line regimes), binary64, against the oracle's rules: 1e-10 of the largest value."""
    wl = W.starfish_domain()
    curves = G.make_curves(wl.curves)
    A = bie.nystrom_matrix(curves, wl.alpha)
    bnd = mh.Boundary(ctx, wl.curves, alpert_order=8)
    rng = np.random.default_rng(6)
    r = np.sqrt(rng.uniform(0.0, 0.95, 40))
    th = rng.uniform(0, 2 * np.pi, 40)
    pts = [np.stack([r * np.cos(th), r * np.sin(th)], axis=1)]
    for c in curves:
        hs = c.speed.mean() * c.h
        for j in rng.choice(c.n, 2, replace=False):
            for d in (3.0, 0.5, 0.1):
                for sgn in (1.0, -1.0):   # the side inside Omega is kept below
                    pts.append((c.nodes[j] + sgn * d * hs * c.normal[j])[None, :])
    pts = np.concatenate(pts)
    info = G.classify(curves, pts)
    pts = pts[info.region == -1]
    info = G.classify(curves, pts)
    assert pts.shape[0] > 60
    sigma = rng.standard_normal(bnd.n) * 0.1 + np.cos(np.concatenate([c.t for c in curves]))
    ref = bie.dlp_eval(curves, sigma, wl.alpha, pts, info, A @ sigma)
    got = torch.empty(pts.shape[0], dtype=torch.float64, device="cuda")
    mh.mh_double_layer_apply(ctx, bnd, wl.alpha, torch.tensor(sigma, device="cuda"), got,
                             targets=torch.tensor(pts, device="cuda"))
    assert np.max(np.abs(got.cpu().numpy() - ref)) < 1e-10 * np.max(np.abs(ref))
