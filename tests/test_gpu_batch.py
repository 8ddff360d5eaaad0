"""Parity of the batched solve (sphgrp_batch_*): many independent periodic boxes of
uneven sizes, uniform and clustered, with uneven active fractions, in one call.

Per box the results must be those of the oracle on that box alone: the iterated h a
converged h under the oracle's arithmetic (and equal to the oracle's iterate almost
everywhere), neighbour counts equal, density within 1e-5, accelerations and du/dt
within 1e-4 (relative L2) at the GPU's h / rho / f, the backward within 1e-3.  A CUDA
graph replay must give bit-identical results to the eager call.
"""

import functools

import numpy as np
import pytest

import oracle
from gpu_common import NEFF_TOL
import sphgen

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-5
ACC_TOL = 1e-4
GRAD_TOL = 1e-3
FIELDS = ("h", "rho", "drhodh", "fgrad", "nngb", "acc", "dudt")


@functools.lru_cache(maxsize=None)
def _case():
    b = sphgen.batch(5, 2500, 24000, config=31)
    n = int(b["box_off"][-1])
    b["m32"] = b["m"].astype(np.float32)
    b["vel32"] = b["vel"].astype(np.float32)
    b["u32"] = b["u"].astype(np.float32)
    # inputs of the inactive particles' hydro: the oracle density at their h
    rho0 = np.empty(n, np.float32)
    f0 = np.empty(n, np.float32)
    for k in range(5):
        s = slice(b["box_off"][k], b["box_off"][k + 1])
        ref = oracle.density(b["pos"][s], b["m32"][s].astype(np.float64), b["h0"][s])
        rho0[s] = ref["rho"]
        f0[s] = ref["f"]
    b["rho0"], b["f0"] = rho0, f0
    rng = np.random.default_rng(sphgen.SEED_BASE + 531)
    b["w"] = rng.standard_normal((n, 3)).astype(np.float32)
    b["s"] = rng.standard_normal(n).astype(np.float32)
    return b


class Io:
    """Device arrays of one batch call; reset() restores the inputs in place (the
    pointers stay, as a graph replay needs)."""

    def __init__(self, b, backward=False):
        import torch

        self.torch = torch
        dev = torch.device("cuda:0")
        n = int(b["box_off"][-1])
        t = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=dt)  # noqa: E731
        self.b = b
        self.a = {
            "pos": t(b["pos"]), "m": t(b["m32"]), "vel": t(b["vel32"]), "u": t(b["u32"]),
            "h": t(b["h0"], torch.float64), "active": t(b["active"].astype(np.uint8)),
            "rho": t(b["rho0"]), "drhodh": torch.zeros(n, device=dev), "fgrad": t(b["f0"]),
            "nngb": torch.zeros(n, dtype=torch.int32, device=dev),
            "acc": torch.zeros((n, 3), device=dev), "dudt": torch.zeros(n, device=dev),
        }
        if backward:
            self.a.update({"g_acc": t(b["w"]), "g_rho": t(b["s"]), "g_pos": torch.zeros((n, 3), device=dev),
                           "g_vel": torch.zeros((n, 3), device=dev), "g_m": torch.zeros(n, device=dev)})

    def reset(self):
        b = self.b
        self.a["h"].copy_(self.torch.as_tensor(b["h0"]))
        self.a["rho"].copy_(self.torch.as_tensor(b["rho0"]))
        self.a["fgrad"].copy_(self.torch.as_tensor(b["f0"]))
        for k in ("drhodh", "nngb", "acc", "dudt", "g_pos", "g_vel", "g_m"):
            if k in self.a:
                self.a[k].zero_()

    def host(self):
        return {k: v.cpu().numpy() for k, v in self.a.items()}


@functools.lru_cache(maxsize=None)
def _forward():
    import paper_1810_09898_gb300 as sg

    b = _case()
    B = sg.Batch(b["box_off"], b["box_class"])
    io = Io(b)
    B.run(io.a)
    out = io.host()
    stats = B.stats()
    B.close()
    return out, stats


def _boxes(b):
    for k in range(len(b["box_off"]) - 1):
        yield k, slice(int(b["box_off"][k]), int(b["box_off"][k + 1]))


def test_batch_density_per_box(cuda_device):
    b = _case()
    out, stats = _forward()
    assert stats["walks"] > 0 and stats["pairs"] > 0
    _check_density_per_box(b, out)


def _check_density_per_box(b, out):
    """Every box's active particles against the oracle: h converged by the oracle's own
    arithmetic, counts bit-exact, rho and f within the bars, h equal to the oracle's
    iterate to 1e-5 for 99.9% of them; inactive particles keep their h."""
    for k, s in _boxes(b):
        act = np.flatnonzero(b["active"][s]).astype(np.int32)
        pos, m = b["pos"][s], b["m32"][s].astype(np.float64)
        h = out["h"][s]
        # inactive h untouched
        inact = np.setdiff1d(np.arange(s.stop - s.start), act)
        assert np.array_equal(h[inact], b["h0"][s][inact])
        chk = oracle.density(pos, m, h, targets=act)
        neff = 4.0 * np.pi / 3.0 * h[act] ** 3 * chk["rho"] / m[act]
        assert np.all(np.abs(neff - 64.0) <= NEFF_TOL), k
        assert np.array_equal(out["nngb"][s][act], chk["nngb"]), k
        assert np.max(np.abs(out["rho"][s][act] / chk["rho"] - 1.0)) <= RHO_TOL, k
        assert np.max(np.abs(out["fgrad"][s][act] / chk["f"] - 1.0)) <= 1e-4, k
        href, _ = oracle.density_iterate(pos, m, b["h0"][s].copy(), targets=act)
        close = np.abs(h[act] / href[act] - 1.0) <= 1e-5
        assert close.mean() > 0.999, (k, close.mean())


def test_batch_hydro_per_box(cuda_device):
    b = _case()
    out, _ = _forward()
    for k, s in _boxes(b):
        act = np.flatnonzero(b["active"][s]).astype(np.int32)
        ref = oracle.hydro(b["pos"][s], b["vel32"][s].astype(np.float64), b["m32"][s].astype(np.float64),
                           out["h"][s], out["rho"][s].astype(np.float64), out["fgrad"][s].astype(np.float64),
                           b["u32"][s].astype(np.float64), targets=act)
        acc = out["acc"][s][act]
        assert np.linalg.norm(acc - ref["acc"]) / np.linalg.norm(ref["acc"]) <= ACC_TOL, k
        dudt = out["dudt"][s][act]
        assert np.linalg.norm(dudt - ref["dudt"]) / np.linalg.norm(ref["dudt"]) <= ACC_TOL, k
        inact = np.setdiff1d(np.arange(s.stop - s.start), act)
        assert np.all(out["acc"][s][inact] == 0.0)


def test_batch_matches_single_box_calls(cuda_device):
    """Every box through the single-box entry points at the batch's h gives the same
    density (to FP32 summation order) and hydro forces."""
    import torch

    import paper_1810_09898_gb300 as sg

    b = _case()
    out, _ = _forward()
    dev = torch.device("cuda:0")
    for k, s in _boxes(b):
        nb = s.stop - s.start
        act = torch.as_tensor(np.flatnonzero(b["active"][s]).astype(np.int32), device=dev)
        ctx = sg.Context(nb)
        pos = torch.as_tensor(b["pos"][s], device=dev)
        ctx.sfc_keys_sort(pos)
        ctx.tree_build(pos, torch.as_tensor(b["m32"][s], device=dev))
        h = torch.as_tensor(out["h"][s], device=dev)
        rho, drho, f = (torch.zeros(nb, device=dev) for _ in range(3))
        nn = torch.zeros(nb, dtype=torch.int32, device=dev)
        ctx.density(act, h, 0, sg.GROUPED, 16, rho, drho, f, nn)
        a = act.cpu().numpy()
        assert np.array_equal(nn.cpu().numpy()[a], out["nngb"][s][a])
        assert np.max(np.abs(rho.cpu().numpy()[a] / out["rho"][s][a] - 1.0)) <= 1e-6
        acc = torch.zeros((nb, 3), device=dev)
        dudt = torch.zeros(nb, device=dev)
        ctx.hydro_force(act, h, torch.as_tensor(out["rho"][s], device=dev), torch.as_tensor(out["fgrad"][s], device=dev),
                        torch.as_tensor(b["vel32"][s], device=dev), torch.as_tensor(b["u32"][s], device=dev),
                        sg.GROUPED, 16, acc, dudt)
        ra = acc.cpu().numpy()[a]
        assert np.linalg.norm(ra - out["acc"][s][a]) <= 1e-6 * np.linalg.norm(ra)
        ctx.close()


def test_batch_graph_replay_is_bit_identical(cuda_device):
    import paper_1810_09898_gb300 as sg

    b = _case()
    B = sg.Batch(b["box_off"], b["box_class"])
    io = Io(b, backward=True)
    B.run(io.a, backward=True)
    eager = io.host()
    for rep in range(3):
        io.reset()
        B.run(io.a, backward=True, graph=True)
        st = B.stats()
        assert st["iterations"] == (1 if rep > 0 else 0)
        got = io.host()
        for key in FIELDS + ("g_pos", "g_vel", "g_m"):
            assert np.array_equal(got[key], eager[key]), (rep, key)
    # a forward-only call with the same io is another graph
    io.reset()
    B.run(io.a, graph=True)
    assert B.stats()["iterations"] == 0
    fwd = io.host()
    for key in FIELDS:
        assert np.array_equal(fwd[key], eager[key]), key
    B.close()


def test_batch_backward_per_box(cuda_device):
    import paper_1810_09898_gb300 as sg

    b = _case()
    B = sg.Batch(b["box_off"], b["box_class"])
    io = Io(b, backward=True)
    B.run(io.a, backward=True)
    out = io.host()
    B.close()
    for k, s in _boxes(b):
        _, ox, ov, om = oracle.loss_grad(b["pos"][s], b["vel32"][s].astype(np.float64),
                                         b["m32"][s].astype(np.float64), b["u32"][s].astype(np.float64),
                                         out["h"][s], b["w"][s].astype(np.float64), b["s"][s].astype(np.float64))
        for got, ref, what in ((out["g_pos"][s], ox, "x"), (out["g_vel"][s], ov, "v"), (out["g_m"][s], om, "m")):
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            worst = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err <= GRAD_TOL and worst <= GRAD_TOL, (k, what, err, worst)


def test_batch_tune_and_config(cuda_device):
    import paper_1810_09898_gb300 as sg

    b = _case()
    B = sg.Batch(b["box_off"], b["box_class"])
    io = Io(b)
    B.tune(io.a)
    for cls in (0, 1):
        cfg = B.get_config(cls)
        assert cfg["group_size"] in (4, 8, 16, 32, 64)
        assert cfg["max_slices"] in (1, 2, 4)
        assert cfg["group_split"] in (1.5, 2.0, 4.0)
        assert cfg["leaf_size"] in (0, 8, 12, 24, 32)
    # a tuned run is still a correct run, by the oracle
    io.reset()
    B.run(io.a, graph=True)
    _check_density_per_box(b, io.host())
    for cls in (0, 1):
        cfg = B.get_config(cls)
        assert cfg["tuned_pass_ms"] > 0.0 and cfg["tuned_members"] == int(
            sum(b["active"][b["box_off"][k]:b["box_off"][k + 1]].sum() for k in range(5) if b["box_class"][k] == cls))
    B.set_config(1, 8, 2, 2.0)
    assert B.get_config(1) == {"group_size": 8, "max_slices": 2, "group_split": 2.0, "leaf_size": 0,
                               "tuned_pass_ms": 0.0, "tuned_members": 0}
    # per-class leaf sizes: the forest of each class's boxes splits at its own bucket size,
    # and the run still agrees with the oracle box by box
    B.set_config(0, 16, 2, 2.0, leaf_size=8)
    B.set_config(1, 8, 4, 2.0, leaf_size=32)
    assert B.get_config(0)["leaf_size"] == 8 and B.get_config(1)["leaf_size"] == 32
    io.reset()
    B.run(io.a)
    _check_density_per_box(b, io.host())
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        B.set_config(1, 0, 2, 2.0)
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        B.set_config(1, 16, 3, 2.0)
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        B.set_config(1, 16, 2, 2.0, leaf_size=4)
    B.close()


def test_batch_rejects_bad_input(cuda_device):
    import torch

    import paper_1810_09898_gb300 as sg

    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        sg.Batch([0, 10, 10, 30])
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        sg.Batch([0, 10, 30], box_class=[0, 9])
    b = _case()
    B = sg.Batch(b["box_off"], b["box_class"])
    io = Io(b)
    io.a["pos"][7, 1] = 1.5
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        B.run(io.a)
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        B.run({k: v for k, v in io.a.items() if k != "acc"})
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        B.run(io.a, backward=True)   # no g_acc
    B.close()
    torch.cuda.synchronize()


def test_batch_single_box_equals_context(cuda_device):
    """One box through the batch call gives the single-box entry points' results."""
    import torch

    import paper_1810_09898_gb300 as sg

    d = sphgen.make("clustered", 12000, config=33)
    n = 12000
    dev = torch.device("cuda:0")
    m32 = d["m"].astype(np.float32)
    b = {"pos": d["pos"], "m32": m32, "vel32": d["vel"].astype(np.float32), "u32": d["u"].astype(np.float32),
         "h0": np.full(n, d["h0"]), "active": np.ones(n, bool), "rho0": np.zeros(n, np.float32),
         "f0": np.ones(n, np.float32), "box_off": np.array([0, n])}
    B = sg.Batch(b["box_off"], [1])
    io = Io(b)
    B.run(io.a)
    out = io.host()
    B.close()
    ctx = sg.Context(n)
    pos = torch.as_tensor(d["pos"], device=dev)
    ctx.sfc_keys_sort(pos)
    ctx.tree_build(pos, torch.as_tensor(m32, device=dev))
    h = torch.as_tensor(out["h"], device=dev)
    act = torch.arange(n, dtype=torch.int32, device=dev)
    rho, drho, f = (torch.zeros(n, device=dev) for _ in range(3))
    nn = torch.zeros(n, dtype=torch.int32, device=dev)
    ctx.density(act, h, 0, sg.GROUPED, 16, rho, drho, f, nn)
    assert np.array_equal(nn.cpu().numpy(), out["nngb"])
    assert np.max(np.abs(rho.cpu().numpy() / out["rho"] - 1.0)) <= 1e-6
    ref = oracle.density(d["pos"], m32.astype(np.float64), out["h"])
    neff = 4.0 * np.pi / 3.0 * out["h"] ** 3 * ref["rho"] / m32
    assert np.all(np.abs(neff - 64.0) <= NEFF_TOL)
    ctx.close()


def test_batch_inactive_boxes_and_no_actives(cuda_device):
    """A box without active particles is left untouched; a call with none at all does
    nothing and succeeds."""
    import paper_1810_09898_gb300 as sg

    b = dict(_case())
    act = b["active"].copy()
    s1 = slice(int(b["box_off"][1]), int(b["box_off"][2]))
    act[s1] = False
    b["active"] = act
    B = sg.Batch(b["box_off"], b["box_class"])
    io = Io(b)
    B.run(io.a)
    out = io.host()
    assert np.array_equal(out["h"][s1], b["h0"][s1])
    assert np.all(out["acc"][s1] == 0.0) and np.all(out["nngb"][s1] == 0)
    s0 = slice(int(b["box_off"][0]), int(b["box_off"][1]))
    assert np.all(out["nngb"][s0][b["active"][s0]] > 0)
    b["active"] = np.zeros_like(act)
    io2 = Io(b)
    B.run(io2.a)
    out2 = io2.host()
    assert np.array_equal(out2["h"], b["h0"]) and np.all(out2["acc"] == 0.0)
    assert B.stats()["pairs"] == 0
    B.close()


def test_batch_many_small_boxes(cuda_device):
    """300 boxes: the box sort takes two radix passes (more than 256 boxes) and the walks
    start at the boxes' roots (no start tables for more than 256 boxes); sampled boxes
    match the oracle."""
    import paper_1810_09898_gb300 as sg

    b = sphgen.batch(300, 1500, 3000, config=35, frac_min=0.5, frac_max=1.0)
    n = int(b["box_off"][-1])
    b["m32"] = b["m"].astype(np.float32)
    b["vel32"] = b["vel"].astype(np.float32)
    b["u32"] = b["u"].astype(np.float32)
    b["rho0"] = np.ones(n, np.float32)
    b["f0"] = np.ones(n, np.float32)
    B = sg.Batch(b["box_off"], b["box_class"])
    io = Io(b)
    B.run(io.a)
    out = io.host()
    B.close()
    for k in (0, 137, 299):
        s = slice(int(b["box_off"][k]), int(b["box_off"][k + 1]))
        act = np.flatnonzero(b["active"][s]).astype(np.int32)
        m = b["m32"][s].astype(np.float64)
        chk = oracle.density(b["pos"][s], m, out["h"][s], targets=act)
        neff = 4.0 * np.pi / 3.0 * out["h"][s][act] ** 3 * chk["rho"] / m[act]
        assert np.all(np.abs(neff - 64.0) <= NEFF_TOL), k
        assert np.array_equal(out["nngb"][s][act], chk["nngb"]), k
        assert np.max(np.abs(out["rho"][s][act] / chk["rho"] - 1.0)) <= RHO_TOL, k
