"""Parity at the benchmark's full size and launch configuration: clustered N = 2^24
(half uniform, half in 256 Plummer spheres), grouped form with g = 16 and the default
parameters, as bench.py times it.  A cold density iteration from the uniform-density
guess, then the timed step's work: h scattered by exp(0.05 N(0,1)) and iterated back,
hydro forces, and the velocity divergence and curl.

Keys and order are compared in full (bit-exact).  The pair sums are compared on a
seeded sample of particles, which the oracle computes one by one at the GPU's h (and,
for the hydro and velocity loops, with the GPU's rho and f of every particle as
inputs): neighbour counts bit-exact, rho rel <= 1e-5 with the GPU's h a converged h
under the oracle's own arithmetic, accelerations, du/dt, div v and curl v rel-L2 <=
1e-4 over the sample.  The same at 10% active (key-order runs of mean length 32).
"""

import numpy as np
import pytest

import oracle
import sphgen
from gpu_common import NEFF_TOL, Gpu, active_runs

pytestmark = pytest.mark.gpu

N = 1 << 24
G = 16
SAMPLE = 2048
RHO_TOL = 1e-5
ACC_TOL = 1e-4


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def full(cuda_device):
    d = sphgen.make("clustered", N, config=3)
    d["m32"] = d["m"].astype(np.float32)
    d["vel32"] = d["vel"].astype(np.float32)
    d["u32"] = d["u"].astype(np.float32)
    gpu = Gpu(d["pos"], d["m32"])
    act = np.arange(N, dtype=np.int32)
    cold = gpu.density(act, np.full(N, d["h0"]), 1, 1, G)
    yield d, gpu, cold
    gpu.ctx.close()


def _check_density(d, out, sample):
    m = d["m32"].astype(np.float64)
    chk = oracle.density(d["pos"], m, out["h"], targets=sample)
    assert np.array_equal(out["nngb"][sample], chk["nngb"])
    rel = np.abs(out["rho"][sample] / chk["rho"] - 1.0)
    assert rel.max() <= RHO_TOL, (int(sample[np.argmax(rel)]), float(rel.max()))
    neff = 4.0 * np.pi / 3.0 * out["h"][sample] ** 3 * chk["rho"] / m[sample]
    assert np.all(np.abs(neff - 64.0) <= NEFF_TOL)


def _check_hydro(d, h, rho32, f32, hyd, sample):
    ref = oracle.hydro(d["pos"], d["vel32"].astype(np.float64), d["m32"].astype(np.float64), h,
                       rho32.astype(np.float64), f32.astype(np.float64), d["u32"].astype(np.float64),
                       targets=sample)
    assert np.array_equal(hyd["nngb"][sample], ref["nngb"])
    assert _rel_l2(hyd["acc"][sample], ref["acc"]) <= ACC_TOL
    assert _rel_l2(hyd["dudt"][sample], ref["dudt"]) <= ACC_TOL


def test_fullsize_keys_and_order_bit_exact(full):
    d, gpu, _ = full
    keys = oracle.hilbert_keys(d["pos"])
    perm = oracle.stable_order(keys)
    assert np.array_equal(gpu.perm.cpu().numpy(), perm)
    assert np.array_equal(gpu.keys.cpu().numpy().view(np.uint64), keys[perm])


def test_fullsize_step_all_active(full):
    d, gpu, cold = full
    torch = gpu.torch
    act = np.arange(N, dtype=np.int32)
    rng = np.random.default_rng(sphgen.SEED_BASE + 240)
    out = gpu.density(act, cold["h"] * np.exp(0.05 * rng.standard_normal(N)), 1, 1, G)
    hyd = gpu.hydro(act, out["h"], out["rho"], out["f"], d["vel32"], d["u32"], 1, G)
    divv = torch.zeros(N, dtype=torch.float32, device=gpu.dev)
    curl = torch.zeros((N, 3), dtype=torch.float32, device=gpu.dev)
    gpu.ctx.velocity_derivs(gpu.t(act, torch.int32), gpu.t(out["h"], torch.float64), gpu.t(out["rho"]),
                            gpu.t(d["vel32"]), G, divv, curl)
    sample = np.sort(rng.choice(N, SAMPLE, replace=False)).astype(np.int32)
    _check_density(d, out, sample)
    _check_hydro(d, out["h"], out["rho"], out["f"], hyd, sample)
    rdiv, rcurl = oracle.velocity_derivs(d["pos"], d["vel32"].astype(np.float64), d["m32"].astype(np.float64),
                                         out["h"], out["rho"].astype(np.float64), targets=sample)
    assert _rel_l2(divv.cpu().numpy()[sample], rdiv) <= ACC_TOL
    assert _rel_l2(curl.cpu().numpy()[sample], rcurl) <= ACC_TOL


def test_fullsize_step_ten_percent_active(full):
    d, gpu, cold = full
    act = active_runs(N, 0.1, 241, gpu.perm.cpu().numpy())
    rng = np.random.default_rng(sphgen.SEED_BASE + 242)
    h = cold["h"].copy()
    h[act] *= np.exp(0.05 * rng.standard_normal(len(act)))
    out = gpu.density(act, h, 1, 1, G)
    inactive = np.setdiff1d(np.arange(N), act)
    assert np.array_equal(out["h"][inactive], cold["h"][inactive])
    assert np.all(out["rho"][inactive] == 0.0)
    # neighbours outside the active set keep their cold-start density and f
    is_act = np.zeros(N, dtype=bool)
    is_act[act] = True
    rho = np.where(is_act, out["rho"], cold["rho"]).astype(np.float32)
    f = np.where(is_act, out["f"], cold["f"]).astype(np.float32)
    hyd = gpu.hydro(act, out["h"], rho, f, d["vel32"], d["u32"], 1, G)
    sample = np.sort(rng.choice(act, SAMPLE // 2, replace=False)).astype(np.int32)
    _check_density(d, out, sample)
    _check_hydro(d, out["h"], rho, f, hyd, sample)
    assert np.all(hyd["acc"][inactive] == 0.0)


# ---------------------------------------------------------------- batched boxes at full size

BATCH_FIELDS = ("h", "rho", "drhodh", "fgrad", "nngb", "acc", "dudt")


@pytest.fixture(scope="module")
def boxes(cuda_device):
    """The batched workload as bench.py times it: 96 boxes (N per box log-uniform in
    [1e4, 2e6], about 41.5 M particles), a cold all-active step, the active sets and the
    scattered h, the per-class autotuner, then one eager step and the same step replayed
    from the captured graph."""
    import torch

    import paper_1810_09898_gb300 as sg

    b = sphgen.batch(96, 10_000, 2_000_000, config=5)
    n = int(b["box_off"][-1])
    dev = torch.device("cuda:0")
    t = lambda x, dt=None: torch.from_numpy(np.ascontiguousarray(x)).to(dev, dtype=dt)  # noqa: E731
    f32 = dict(dtype=torch.float32, device=dev)
    io = {"pos": t(b["pos"]), "m": t(b["m"], torch.float32), "vel": t(b["vel"], torch.float32),
          "u": t(b["u"], torch.float32), "h": t(b["h0"]), "active": None,
          "rho": torch.zeros(n, **f32), "drhodh": torch.zeros(n, **f32), "fgrad": torch.ones(n, **f32),
          "nngb": torch.zeros(n, dtype=torch.int32, device=dev), "acc": torch.zeros((n, 3), **f32),
          "dudt": torch.zeros(n, **f32)}
    B = sg.Batch(b["box_off"], b["box_class"])
    B.run(io)
    io["active"] = t(b["active"].astype(np.uint8))
    rng = np.random.default_rng(sphgen.SEED_BASE + 243)
    hc = io["h"].cpu().numpy()
    h_init = t(np.where(b["active"], hc * np.exp(0.05 * rng.standard_normal(n)), hc))
    io["h"].copy_(h_init)
    B.tune(io)
    io["h"].copy_(h_init)
    B.run(io)
    eager = {k: io[k].cpu().numpy() for k in BATCH_FIELDS}
    for _ in range(2):   # capture, then replay
        io["h"].copy_(h_init)
        B.run(io, graph=True)
    graph = {k: io[k].cpu().numpy() for k in BATCH_FIELDS}
    B.close()
    yield b, eager, graph


def test_batch_fullsize_graph_replay_bit_identical(boxes):
    _, eager, graph = boxes
    for k in BATCH_FIELDS:
        assert np.array_equal(eager[k], graph[k]), k


def test_batch_fullsize_sampled_boxes(boxes):
    b, _, out = boxes
    sizes = np.diff(b["box_off"])
    cls = b["box_class"]
    picks = {int(np.argmax(sizes)),
             int(np.flatnonzero(cls == 0)[np.argmin(sizes[cls == 0])]),
             int(np.flatnonzero(cls == 1)[np.argmin(sizes[cls == 1])])}
    rng = np.random.default_rng(sphgen.SEED_BASE + 244)
    for k in sorted(picks):
        s = slice(int(b["box_off"][k]), int(b["box_off"][k + 1]))
        act = np.flatnonzero(b["active"][s])
        sample = np.sort(rng.choice(act, min(512, len(act)), replace=False)).astype(np.int32)
        pos, m = b["pos"][s], b["m"][s].astype(np.float32).astype(np.float64)
        h = out["h"][s]
        chk = oracle.density(pos, m, h, targets=sample)
        assert np.array_equal(out["nngb"][s][sample], chk["nngb"]), k
        assert np.max(np.abs(out["rho"][s][sample] / chk["rho"] - 1.0)) <= RHO_TOL, k
        neff = 4.0 * np.pi / 3.0 * h[sample] ** 3 * chk["rho"] / m[sample]
        assert np.all(np.abs(neff - 64.0) <= NEFF_TOL), k
        ref = oracle.hydro(pos, b["vel"][s].astype(np.float32).astype(np.float64), m, h,
                           out["rho"][s].astype(np.float64), out["fgrad"][s].astype(np.float64),
                           b["u"][s].astype(np.float32).astype(np.float64), targets=sample)
        assert _rel_l2(out["acc"][s][sample], ref["acc"]) <= ACC_TOL, k
        assert _rel_l2(out["dudt"][s][sample], ref["dudt"]) <= ACC_TOL, k


# ---------------------------------------------------------------- group-size sweep at full size

def test_group_size_sweep_fullsize(cuda_device):
    """The group-size sweep's workload at its full size: clustered N = 2^21, 20% active
    in key-order runs, h scattered by exp(0.05 N(0,1)) and iterated, for every group
    size of the sweep; sampled actives against the oracle at each g's h, and hydro at
    g = 16."""
    n = 1 << 21
    d = sphgen.make("clustered", n, config=2)
    m32 = d["m"].astype(np.float32)
    gpu = Gpu(d["pos"], m32)
    cold = gpu.density(np.arange(n, dtype=np.int32), np.full(n, d["h0"]), 1, 1, 16)
    act = active_runs(n, 0.2, 245, gpu.perm.cpu().numpy())
    rng = np.random.default_rng(sphgen.SEED_BASE + 246)
    h = cold["h"].copy()
    h[act] *= np.exp(0.05 * rng.standard_normal(len(act)))
    sample = np.sort(rng.choice(act, 512, replace=False)).astype(np.int32)
    dd = {"pos": d["pos"], "m32": m32}
    for g in (1, 4, 8, 16, 32, 64, 128):
        out = gpu.density(act, h, 1, 1, g)
        _check_density(dd, out, sample)
        if g == 16:
            is_act = np.zeros(n, dtype=bool)
            is_act[act] = True
            rho = np.where(is_act, out["rho"], cold["rho"]).astype(np.float32)
            f = np.where(is_act, out["f"], cold["f"]).astype(np.float32)
            dd.update(vel32=d["vel"].astype(np.float32), u32=d["u"].astype(np.float32))
            hyd = gpu.hydro(act, out["h"], rho, f, dd["vel32"], dd["u32"], 1, g)
            _check_hydro(dd, out["h"], rho, f, hyd, sample)
    gpu.ctx.close()
