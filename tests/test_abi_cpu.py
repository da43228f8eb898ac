"""The C ABI library loads without a GPU and exports every declared symbol;
argument validation that precedes any device work answers on the CPU."""
import ctypes as C
import glob
import os
import re

import pytest

from tests.helpers import ROOT


@pytest.fixture(scope="module")
def built():
    from paper_1511_06103_gb300 import build
    build.build()
    from paper_1511_06103_gb300 import binding
    return binding


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["crf_create", "crf_destroy", "crf_set_unary", "crf_set_pairwise", "mf_iterate",
              "mf_free_energy", "mf_marginals", "mf_lipschitz", "crf_error_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings_and_version(built):
    assert "proxmf" in built.crf_version()
    for code in built.STATUS:
        assert built.error_string(code) not in ("", "?")


@pytest.mark.parametrize("field,value", [("n_labels", 0), ("n_labels", 33), ("batch", 0),
                                         ("height", 0), ("width", -3), ("topology", 9),
                                         ("precision", 5)])
def test_create_rejects_bad_descriptors(built, field, value):
    d = built.crf_desc(built.CRF_GRID4, 3, 1, built.CRF_FP32, 8, 8, None)
    setattr(d, field, value)
    with pytest.raises(built.ProxMFError) as e:
        built.crf_create(d)
    assert e.value.status == -1


def test_null_handle_is_invalid(built):
    with pytest.raises(built.ProxMFError) as e:
        built.mf_free_energy(None, None)
    assert e.value.status == -1
    built.crf_destroy(None)     # accepted
