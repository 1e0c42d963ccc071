"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rnmf.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "rnmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(rnmf_\w+|rnmf)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_02037_gb300 import build
    build.build()
    import paper_1711_02037_gb300 as pkg
    return pkg.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rnmf", "rnmf_hals", "rnmf_qb", "rnmf_sweeps", "rnmf_create", "rnmf_destroy", "rnmf_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    import paper_1711_02037_gb300 as pkg
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in pkg.SIGNATURES, f"binding lacks {name}"


def test_null_context_is_rejected_without_a_gpu(lib):
    import paper_1711_02037_gb300 as pkg
    o = pkg.default_opts()
    assert o.precision == 0 and o.gram_mode == 0 and o.track_every == 0
    # the last field of rnmf_opts: the struct the library fills ends where the binding's does
    assert o.sweep_products == pkg.SWEEP_FP32 and pkg.Opts.sweep_products.offset + 4 <= ctypes.sizeof(pkg.Opts)
    st = lib.rnmf(None, None, 10, 10, 10, 2, 1, 0, 1, 0, None, None, None, None)
    assert st == 1  # RNMF_EINVAL
    assert lib.rnmf_hals(None, None, 10, 10, 10, 2, 1, 0, None, None, None, None) == 1
    assert lib.rnmf_destroy(None) == 1


def test_compiled_for_sm_103a_only():
    from paper_1711_02037_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
