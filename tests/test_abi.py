"""The C-ABI library loads and exports every symbol include/vie.h declares.
No compute call: these run without a GPU."""
import os
import re

import pytest

import paper_1610_00835_gb300 as P
from paper_1610_00835_gb300 import vie as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vie.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                                 text, flags=re.M)) - {"if", "while"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("vie_create", "vie_destroy", "vie_apply", "vie_solve_gmres", "ert_sweep"):
        assert want in names


def test_library_exports_every_declared_symbol():
    L = P.load()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in B.SIGNATURES, f"binding lacks {name}"


def test_version_and_error_string():
    assert "sm_103a" in P.vie_version()
    assert isinstance(P.vie_last_error(), str)


def test_invalid_arguments_rejected_before_device_use():
    with pytest.raises(P.VieError) as e:
        P.vie_create(4, 8, [1.0] * 64, [0.5] * 64)
    assert e.value.status == B.VIE_ERR_INVALID_ARG
    with pytest.raises(P.VieError) as e:
        P.vie_create(2, 8, [1.0] * 64, [0.5] * 64, steps=0)
    assert e.value.status == B.VIE_ERR_INVALID_ARG
