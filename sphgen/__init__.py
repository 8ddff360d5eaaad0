"""Seeded synthetic particle sets for the SPH neighbour-search workloads.

This module only draws random numbers and lays them out.  It contains none of the
method's arithmetic (no space-filling-curve keys, no smoothing kernel, no neighbour
test), so that both the FP64 oracle and the CUDA path can take their inputs from it
without sharing any of the computation they are compared on.

Workloads (all in a periodic unit cube, coordinates in [0, 1)):

* ``uniform``   -- N positions uniform random.
* ``clustered`` -- half uniform, half in 256 Plummer spheres: centres uniform, scale
  radius log-uniform in [0.002, 0.02], member counts from a Pareto(alpha=1.5) draw
  normalised to N/2 by largest remainder; Plummer radii r = a / sqrt(u^(-2/3) - 1),
  redrawn while r > 0.25 so that the minimum-image convention stays valid; isotropic
  directions; positions wrapped into the unit cube.
* velocities Gaussian (sigma 0.1 per component), specific internal energy
  log-normal (mu 0, sigma 1), equal masses m = 1/N.
* active sets as runs along the sorted (space-filling-curve) order: run starts uniform
  over the N ranks, run lengths geometric with a given mean, drawn until the requested
  number of ranks is marked (the last run truncated).  The mask is returned in *rank*
  space; the caller maps ranks to particles with its own sort permutation.

The paper's own test data (a Magneticum cosmological box) is not available; these
sets stand in for it with the particle counts, clustering and active fractions of the
benchmark configurations.
"""

from __future__ import annotations

import math

import numpy as np

SEED_BASE = 18100989
NNGB = 64.0
NNGB_TOL = 2.0
GAMMA = 5.0 / 3.0
ALPHA_VISC = 1.0
BETA_VISC = 2.0
EPS_VISC = 0.01


def rng_for(config: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config + 1000 * salt))


def h_initial(n: int, nngb: float = NNGB) -> float:
    """Initial smoothing length of the uniform configuration, (3 Nngb / (4 pi N))^(1/3)."""
    return (3.0 * nngb / (4.0 * math.pi * n)) ** (1.0 / 3.0)


def _wrap_unit(p: np.ndarray) -> np.ndarray:
    p = np.mod(p, 1.0)
    p[p >= 1.0] = 0.0  # np.mod can round a tiny negative value up to exactly 1.0
    return p


def uniform_positions(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.random((n, 3))


def _largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    share = weights / weights.sum() * total
    counts = np.floor(share).astype(np.int64)
    short = total - int(counts.sum())
    if short > 0:
        order = np.argsort(-(share - counts), kind="stable")
        counts[order[:short]] += 1
    return counts


def plummer_positions(n: int, rng: np.random.Generator, n_spheres: int = 256,
                      a_lo: float = 0.002, a_hi: float = 0.02, alpha: float = 1.5,
                      r_max: float = 0.25) -> np.ndarray:
    centres = rng.random((n_spheres, 3))
    scale = np.exp(rng.uniform(math.log(a_lo), math.log(a_hi), n_spheres))
    weights = rng.pareto(alpha, n_spheres) + 1.0
    counts = _largest_remainder(weights, n)
    out = np.empty((n, 3))
    pos = 0
    for k in range(n_spheres):
        c = int(counts[k])
        if c == 0:
            continue
        r = np.empty(c)
        todo = np.arange(c)
        while todo.size:
            u = rng.random(todo.size)
            u = np.where(u <= 0.0, 0.5, u)
            rr = scale[k] / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
            ok = np.isfinite(rr) & (rr <= r_max)
            r[todo[ok]] = rr[ok]
            todo = todo[~ok]
        cz = rng.uniform(-1.0, 1.0, c)
        phi = rng.uniform(0.0, 2.0 * math.pi, c)
        sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
        d = np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)
        out[pos:pos + c] = centres[k] + r[:, None] * d
        pos += c
    return _wrap_unit(out)


def clustered_positions(n: int, rng: np.random.Generator) -> np.ndarray:
    nu = n // 2
    p = np.concatenate([uniform_positions(nu, rng), plummer_positions(n - nu, rng)])
    return p[rng.permutation(n)]


def active_rank_mask(n: int, frac: float, mean_len: float, rng: np.random.Generator) -> np.ndarray:
    """Boolean mask over sorted ranks: geometric-length runs until floor(frac*n) are set."""
    target = int(math.floor(frac * n))
    mask = np.zeros(n, dtype=bool)
    if target >= n:
        mask[:] = True
        return mask
    marked = 0
    p = 1.0 / mean_len
    while marked < target:
        starts = rng.integers(0, n, 4096)
        lens = rng.geometric(p, 4096)
        for s, ln in zip(starts.tolist(), lens.tolist()):
            e = min(n, s + ln)
            seg = mask[s:e]
            new = np.flatnonzero(~seg)
            if new.size == 0:
                continue
            need = target - marked
            if new.size > need:
                new = new[:need]
            seg[new] = True
            marked += new.size
            if marked >= target:
                break
    return mask


def make(kind: str, n: int, config: int = 1, seed_salt: int = 0, with_hydro: bool = True) -> dict:
    """One particle set: positions (n,3) f64, masses, velocities, internal energies, h0."""
    rng = rng_for(config, seed_salt)
    if kind == "uniform":
        pos = uniform_positions(n, rng)
    elif kind == "clustered":
        pos = clustered_positions(n, rng)
    else:
        raise ValueError(kind)
    out = {
        "pos": np.ascontiguousarray(pos),
        "m": np.full(n, 1.0 / n),
        "h0": h_initial(n),
        "kind": kind,
        "n": n,
    }
    if with_hydro:
        out["vel"] = rng.normal(0.0, 0.1, (n, 3))
        out["u"] = rng.lognormal(0.0, 1.0, n)
    return out


def lattice(n_side: int) -> np.ndarray:
    """A simple cubic lattice of n_side^3 points with spacing 1/n_side (offset half a cell)."""
    g = (np.arange(n_side) + 0.5) / n_side
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def batch(nbox: int, n_min: int, n_max: int, config: int = 5, seed_salt: int = 0,
          frac_min: float = 0.01, frac_max: float = 1.0) -> dict:
    """Many independent periodic boxes, concatenated (the batched workload).

    Per box: N log-uniform in [n_min, n_max], uniform or clustered by a fair coin,
    active fraction uniform in [frac_min, frac_max] (each particle active with that
    probability, at least one per box).  Box k's particles are the rows
    box_off[k] .. box_off[k+1] of every array; box_class is 0 for uniform, 1 for
    clustered; h0 is each box's own initial guess, per particle."""
    rng = rng_for(config, seed_salt)
    sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), nbox)).astype(np.int64)
    kinds = np.where(rng.random(nbox) < 0.5, "uniform", "clustered")
    fracs = rng.uniform(frac_min, frac_max, nbox)
    parts = []
    for k in range(nbox):
        d = make(str(kinds[k]), int(sizes[k]), config=config, seed_salt=1000 * (seed_salt + 1) + k)
        act = rng.random(int(sizes[k])) < fracs[k]
        if not act.any():
            act[rng.integers(0, int(sizes[k]))] = True
        d["active"] = act
        parts.append(d)
    box_off = np.zeros(nbox + 1, dtype=np.int64)
    box_off[1:] = np.cumsum(sizes)
    cat = lambda key: np.concatenate([p[key] for p in parts])  # noqa: E731
    return {
        "pos": np.ascontiguousarray(cat("pos")),
        "m": cat("m"),
        "vel": cat("vel"),
        "u": cat("u"),
        "h0": np.concatenate([np.full(p["n"], p["h0"]) for p in parts]),
        "active": cat("active"),
        "box_off": box_off,
        "box_class": (kinds == "clustered").astype(np.int32),
        "kinds": kinds,
        "fracs": fracs,
    }
