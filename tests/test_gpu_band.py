"""Adversarial pair decisions at the smoothing-length boundary (Sec. 1.1: a neighbour is
closer than h, so r = h is excluded), GPU against the FP64 oracle through the C ABI.

The GPU decides pairs in FP32 on centre-relative coordinates and re-decides those whose
FP32 r^2 lies in the proven error band around the threshold from the FP64 positions.
These inputs put pairs exactly on the boundary and one FP64 ulp either side of it:

* positions on a 2^-20 grid, so that a partner placed along an axis at a dyadic distance
  d from a particle whose h is d has r^2 == h^2 exactly (excluded), and the neighbouring
  FP64 values of h put it just inside or just outside;
* diagonal partners with h = sqrt(r^2) rounded in FP64, then nudged by one ulp;
* partners across the periodic face (minimum image);
* members far from their group's centre and groups reaching across half the box
  (group size 128 without splitting, over a sparse active set), which take the band's
  |m|^2 term, the wrapped differences and the exact-difference physics.

The bar is the usual one: neighbour sets (sorted lists) and counts bit-exact, density
rel <= 1e-5; the calls must have re-decided pairs in FP64.
"""

import numpy as np
import pytest

import oracle
import sphgen
from gpu_common import Gpu, csr_sorted_lists

pytestmark = pytest.mark.gpu

GRID = 2.0 ** -20


def _boundary_set(seed=20231):
    rng = np.random.default_rng(seed)
    n0 = 6000
    pos = np.floor(sphgen.clustered_positions(n0, rng) / GRID) * GRID
    h = np.floor(rng.uniform(0.05, 0.15, n0) / GRID) * GRID
    extra, extra_h = [], []
    planted = []
    # axis-aligned partners at exactly h (dyadic), some across the periodic face
    idx = rng.choice(n0, 900, replace=False)
    for t, i in enumerate(idx):
        ax = rng.integers(3)
        sign = 1.0 if rng.random() < 0.5 else -1.0
        p = pos[i].copy()
        if t % 5 == 0:
            # put i next to the face the partner crosses
            p[ax] = (rng.integers(0, 64) * GRID) if sign < 0 else 1.0 - (rng.integers(1, 64) * GRID)
            pos[i] = p
        q = p.copy()
        q[ax] = (q[ax] + sign * h[i]) % 1.0
        extra.append(q)
        extra_h.append(h[i])
        planted.append(i)
    # diagonal partners: r^2 exact (dyadic offsets), h = sqrt(r^2) in FP64
    idx2 = rng.choice(np.setdiff1d(np.arange(n0), idx), 600, replace=False)
    for i in idx2:
        off = np.floor(rng.uniform(-0.06, 0.06, 3) / GRID) * GRID
        q = (pos[i] + off) % 1.0
        extra.append(q)
        extra_h.append(h[i])
        r2 = (off[0] * off[0] + off[1] * off[1]) + off[2] * off[2]
        h[i] = np.sqrt(r2)
        planted.append(i)
    pos = np.concatenate([pos, np.array(extra)])
    h = np.concatenate([h, np.array(extra_h)])
    # one FP64 ulp inside, on, or outside the boundary
    planted = np.array(planted)
    nudge = rng.integers(-1, 2, len(planted))
    h[planted[nudge > 0]] = np.nextafter(h[planted[nudge > 0]], np.inf)
    h[planted[nudge < 0]] = np.nextafter(h[planted[nudge < 0]], 0.0)
    assert np.all(pos >= 0.0) and np.all(pos < 1.0) and np.all(h > 0.0) and np.all(h < 0.5)
    m = np.full(len(pos), 1.0 / len(pos), np.float32)
    return pos, h, m, planted


@pytest.fixture(scope="module")
def bset(cuda_device):
    pos, h, m, planted = _boundary_set()
    # the construction does put pairs on the boundary: some r^2 == h^2 exactly
    d = pos[len(pos) - 1500:] - pos[planted]
    d -= np.rint(d)
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    on = r2 == h[planted] * h[planted]
    assert on.sum() > 100, on.sum()
    return pos, h, m, planted


CASES = [  # (mode, g, params, active stride)
    (0, 1, {}, 1),
    (1, 16, {}, 1),
    (1, 32, {"group_centre": 0}, 1),
    (1, 128, {"group_split": 0.0}, 7),     # wide groups: far members, wrapped differences
    (1, 128, {"group_split": 0.0, "group_centre": 0}, 13),
]


@pytest.mark.parametrize("mode,g,params,stride", CASES)
@pytest.mark.parametrize("kind", [oracle.DENSITY, oracle.HYDRO])
def test_boundary_sets_bit_exact(bset, mode, g, params, stride, kind):
    pos, h, m, _ = bset
    G = Gpu(pos, m, **params)
    act = np.arange(0, len(pos), stride, dtype=np.int32)
    got = G.ngb_sets(act, h, kind, mode, g)
    st = G.ctx.stats()
    ref = oracle.ngb_sets(pos, h, act, kind)
    a, b = csr_sorted_lists(*got), csr_sorted_lists(*ref)
    bad = [k for k in range(len(a)) if not np.array_equal(a[k], b[k])]
    assert not bad, f"{len(bad)} sets differ, first: particle {act[bad[0]]}"
    assert st["fp64_retests"] > 0, st
    G.ctx.close()


@pytest.mark.parametrize("mode,g,params,stride", CASES)
def test_boundary_density(bset, mode, g, params, stride):
    pos, h, m, _ = bset
    G = Gpu(pos, m, **params)
    act = np.arange(0, len(pos), stride, dtype=np.int32)
    out = G.density(act, h, 0, mode, g)
    ref = oracle.density(pos, m.astype(np.float64), h)
    assert np.array_equal(out["nngb"][act], ref["nngb"][act])
    rel = np.abs(out["rho"][act] / ref["rho"][act] - 1.0)
    assert rel.max() <= 1e-5, rel.max()
    assert out["stats"]["fp64_retests"] > 0
    G.ctx.close()
