"""CPU-only checks of the C ABI: the library builds, loads, exports every
function that include/*.h declares, and rejects bad arguments on the host
before touching a GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import chaingen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:long\s+long|size_t|int|void|char|double|float)"
                             r"\s*\**\s*(\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_1609_04493_gb300 as rd

    return rd.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rd_model_create", "rd_model_destroy", "rnea_batch", "rnea_batch_host",
                     "rnea_vjp", "aba_batch", "jsiia_batch", "fleet_batch",
                     "rd_plan_total_joints", "rd_last_error", "rd_version"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version(lib):
    assert lib.rd_version() >= 100


def _create(lib, n, M, S, J):
    import paper_1609_04493_gb300.binding as b

    h = ctypes.c_void_p()
    D = ctypes.POINTER(ctypes.c_double)
    rc = lib.rd_model_create(n, M.ctypes.data_as(D) if M is not None else None,
                             S.ctypes.data_as(D) if S is not None else None,
                             J.ctypes.data_as(D) if J is not None else None, ctypes.byref(h))
    return rc, lib.rd_last_error().decode(), h, b


def test_model_create_rejects_bad_input_on_host(lib):
    ch = chaingen.make_chain(4)
    rc, msg, _, _ = _create(lib, 0, ch.M, ch.S, ch.inertia)
    assert rc == -3 and "outside" in msg
    rc, msg, _, _ = _create(lib, 129, ch.M, ch.S, ch.inertia)
    assert rc == -3
    rc, msg, _, _ = _create(lib, 4, None, ch.S, ch.inertia)
    assert rc == -1
    S = ch.S.copy()
    S[2, 3:] *= 1.5  # axis not unit
    rc, msg, _, _ = _create(lib, 4, ch.M, S, ch.inertia)
    assert rc == -1 and "axis" in msg
    S = ch.S.copy()
    S[1, :3] += 0.2 * S[1, 3:]  # pitched screw
    rc, msg, _, _ = _create(lib, 4, ch.M, S, ch.inertia)
    assert rc == -1 and "pitch" in msg
    J = ch.inertia.copy()
    J[0, 0] = -1.0
    rc, msg, _, _ = _create(lib, 4, ch.M, ch.S, J)
    assert rc == -1 and "mass" in msg
    J = ch.inertia.copy()
    J[3, 4:7] = [1.0, 1.0, 1.0]
    J[3, 7] = 5.0  # Ixy too large: not positive definite
    rc, msg, _, _ = _create(lib, 4, ch.M, ch.S, J)
    assert rc == -1 and "positive semi-definite" in msg


def test_batch_calls_reject_bad_arguments_on_host(lib):
    P = ctypes.c_void_p
    # null model
    assert lib.rnea_batch(None, 4, 0, P(8), P(8), P(8), P(8), None, 0, None) == -1
    assert "null model" in lib.rd_last_error().decode()
    assert lib.rnea_batch_host(None, 4, 0, P(8), P(8), P(8), P(8), None, 0, None) == -1
    assert lib.rd_model_links(None) == -1


def test_oracle_is_not_linked_by_the_library():
    import paper_1609_04493_gb300 as rd

    so = rd.library_path()
    data = open(so, "rb").read()
    assert b"oracle_rnea" not in data and b"liboracle" not in data
