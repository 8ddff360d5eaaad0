"""The keys + sort entry point that allocates nothing (sphgrp_sfc_keys_sort_static).

It serves callers that may not allocate device memory (a host application owning all
device memory through its own pool, or a path that cannot afford the device
synchronisation of cudaMalloc / cudaFree).  Its output must equal the regular
context-based entry point bit for bit (keys and order are integer results), on two
calls in a row: the static scratch keeps the previous call's contents, so the second
call checks that nothing depends on it.  This file is collected last.
"""

import numpy as np
import pytest

import sphgen

pytestmark = pytest.mark.gpu


def _static_sort(lib, pos):
    """The entry point through the binding's checked wrapper (element types, lengths and
    device of every array are checked before the C call); returns (status, keys, perm)."""
    import torch

    import paper_1810_09898_gb300 as sg

    n = pos.shape[0]
    keys = torch.empty(n, dtype=torch.int64, device=pos.device)
    perm = torch.empty(n, dtype=torch.int32, device=pos.device)
    try:
        sg.sfc_keys_sort_static(pos, keys, perm)
    except sg.SphgrpError as e:
        return e.code, keys, perm
    return 0, keys, perm


def test_static_scratch_sort_equals_context_sort(cuda_device):
    import torch

    import paper_1810_09898_gb300 as sg

    lib = sg.load_library()
    max_n = 1 << 19
    cases = [sphgen.make("clustered", max_n, config=5, with_hydro=False),
             sphgen.make("uniform", 70001, config=6, with_hydro=False)]
    for d in cases:  # two calls in a row, different sizes
        pos = torch.as_tensor(d["pos"], device=cuda_device)
        n = pos.shape[0]
        ctx = sg.Context(n)
        keys_ref = torch.empty(n, dtype=torch.int64, device=cuda_device)
        perm_ref = torch.empty(n, dtype=torch.int32, device=cuda_device)
        ctx.sfc_keys_sort(pos, keys_ref, perm_ref)
        rc, keys, perm = _static_sort(lib, pos)
        assert rc == 0, lib.sphgrp_last_error().decode()
        assert torch.equal(keys, keys_ref)
        assert torch.equal(perm, perm_ref)
        ctx.close()


def test_static_scratch_sort_rejects_oversize_and_bad_input(cuda_device):
    import torch

    import paper_1810_09898_gb300 as sg

    lib = sg.load_library()
    big = torch.zeros(((1 << 19) + 1, 3), dtype=torch.float64, device=cuda_device)
    rc, _, _ = _static_sort(lib, big)
    assert rc == -1 and b"SPHGRP_STATIC_SORT_MAX_N" in lib.sphgrp_last_error()
    bad = torch.tensor([[0.5, 0.5, 1.5], [0.1, 0.2, 0.3]], dtype=torch.float64, device=cuda_device)
    rc, _, _ = _static_sort(lib, bad)
    assert rc == -1
    # a short output array is refused before the C call
    small = torch.zeros((8, 3), dtype=torch.float64, device=cuda_device)
    with pytest.raises(ValueError, match="perm_out"):
        sg.sfc_keys_sort_static(small, torch.empty(8, dtype=torch.int64, device=cuda_device),
                                torch.empty(4, dtype=torch.int32, device=cuda_device))
    # the flag is cleared per call: a good input right after a bad one succeeds
    good = torch.as_tensor(np.random.default_rng(3).random((1000, 3)), device=cuda_device)
    rc, keys, _ = _static_sort(lib, good)
    assert rc == 0
    assert bool((keys[1:] >= keys[:-1]).all())
