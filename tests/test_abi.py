"""CPU checks of the boundary: the library builds, loads, and exports every entry
point declared in include/*.h; the product package never loads the oracle."""

import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(sphgrp_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_1810_09898_gb300.build import build

    return build()


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("sphgrp_sfc_keys_sort", "sphgrp_tree_build", "sphgrp_ngb_search", "sphgrp_density",
                 "sphgrp_hydro_force"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1810_09898_gb300 import binding

    assert set(binding.EXPORTED) <= set(_declared())


def test_library_does_not_link_the_oracle(lib_path):
    out = subprocess.run(["ldd", lib_path], capture_output=True, text=True).stdout
    assert "sphoracle" not in out
    for f in glob.glob(os.path.join(ROOT, "paper_1810_09898_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(f).read()
            assert "import oracle" not in text and "sph_oracle" not in text, f


def test_default_params_and_error_text(lib_path):
    from paper_1810_09898_gb300 import binding

    p = binding.default_params()
    assert p.nngb == 64.0 and p.nngb_tol == 2.0 and p.leaf_size == 16
    lib = binding.load_library()
    # no device needed: argument checks fail before any CUDA call
    h = ctypes.c_void_p()
    assert lib.sphgrp_ctx_create(None, None, 10) == -1
    assert lib.sphgrp_ctx_create(ctypes.byref(h), None, 0) == -1
    assert b"n_max" in lib.sphgrp_last_error()


_CTYPES = {"double": ctypes.c_double, "int": ctypes.c_int, "int64_t": ctypes.c_int64}


def _struct_fields(name):
    """(type, field) of a typedef struct in include/sphgrp.h, in declaration order."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sphgrp.h")).read(), flags=re.S)
    body = re.search(r"typedef struct " + name + r"\s*\{(.*?)\}\s*" + name + ";", text, flags=re.S).group(1)
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.match(r"(const )?([\w]+)\s*(\*?)\s*(\w+)$", decl.replace("* ", " *"))
        assert m, decl
        out.append(("ptr" if m.group(3) else m.group(2), m.group(4)))
    return out


@pytest.mark.parametrize("cname,pyname", [("sphgrp_params", "Params"), ("sphgrp_stats", "Stats"),
                                          ("sphgrp_batch_io", "BatchIO")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes mirrors of the ABI structs have the header's fields, in order and of
    the same C type (a layout mismatch would corrupt every call without a GPU error)."""
    from paper_1810_09898_gb300 import binding

    fields = _struct_fields(cname)
    py = getattr(binding, pyname)._fields_
    assert [f for _, f in fields] == [f for f, _ in py]
    for (ctype, f), (_, pytype) in zip(fields, py):
        if ctype == "ptr":
            assert pytype is ctypes.c_void_p, f
        else:
            assert pytype is _CTYPES[ctype], f


def test_batch_io_rejects_unknown_arrays():
    import torch

    from paper_1810_09898_gb300 import binding

    io = binding.Batch._io({"pos": torch.zeros(3, dtype=torch.float64), "acc": torch.zeros(3)}, 1, cuda=False)
    assert io.pos and io.acc and not io.vel
    with pytest.raises(KeyError):
        binding.Batch._io({"position": torch.zeros(3)}, 1, cuda=False)
    with pytest.raises(ValueError, match="holds 3 elements, needs 6"):
        binding.Batch._io({"acc": torch.zeros(3)}, 2, cuda=False)
    with pytest.raises(TypeError, match="pos must be float64"):
        binding.Batch._io({"pos": torch.zeros(3)}, 1, cuda=False)


def test_arguments_are_checked_before_the_call():
    """Type, density, length and device of every array are checked in the binding, so a
    wrong array never reaches a kernel."""
    import torch

    from paper_1810_09898_gb300 import binding

    ok = torch.zeros((4, 3), dtype=torch.float32)
    assert binding._arg(ok, "vel", "float32", 12, cuda=False).value == ok.data_ptr()
    assert binding._arg(None, "nngb", "int32", 4, optional=True) is None
    with pytest.raises(ValueError, match="required"):
        binding._arg(None, "rho", "float32", 4)
    with pytest.raises(TypeError, match="must be int32"):
        binding._arg(torch.zeros(4, dtype=torch.int64), "active", "int32", 4, cuda=False)
    with pytest.raises(ValueError, match="contiguous"):
        binding._arg(ok.t(), "vel", "float32", 12, cuda=False)
    with pytest.raises(ValueError, match="needs 13"):
        binding._arg(ok, "vel", "float32", 13, cuda=False)
    with pytest.raises(ValueError, match="CUDA device"):
        binding._arg(ok, "vel", "float32", 12)
