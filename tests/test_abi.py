"""The C-ABI library loads and exports every entry point include/salt.h
declares; host-only helpers work without a GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_symbols(headers=None):
    names = set()
    for h in (HEADERS if headers is None else headers):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(salt_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2504_08081_b300 import build as B
    B.build()
    from paper_2504_08081_b300 import _abi
    return _abi.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("salt_init_model", "salt_bandflux", "salt_chi2", "salt_chi2_grad",
              "salt_serve_submit", "salt_serve_poll"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2504_08081_b300 import _abi
    names = declared_symbols([os.path.join(ROOT, "include", "salt.h")])
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert names == set(_abi.EXPORTS), names ^ set(_abi.EXPORTS)
    # the native client library exports what salt_client.h declares
    client = _abi.client()
    cnames = declared_symbols([os.path.join(ROOT, "include", "salt_client.h")])
    assert cnames == set(_abi.CLIENT_EXPORTS), cnames ^ set(_abi.CLIENT_EXPORTS)
    assert all(hasattr(client, n) for n in cnames)
    assert declared_symbols() == names | cnames  # no other header declares entry points


def test_host_helpers_without_gpu(lib):
    from paper_2504_08081_b300 import _abi
    assert lib.salt_status_str(0) == b"ok"
    assert lib.salt_status_str(-1).startswith(b"invalid")
    oo = np.array([0, 3, 3, 10], dtype=np.int64)
    po = np.array([0, 2, 5, 6], dtype=np.int64)
    out = _abi.bandflux_offsets(oo, po)
    np.testing.assert_array_equal(out, [0, 6, 6, 13])
    bad = np.array([0, 3, 2, 10], dtype=np.int64)
    with pytest.raises(_abi.SaltError):
        _abi.bandflux_offsets(bad, po)
    # null context arguments are rejected before any CUDA call
    assert lib.salt_set_option(None, 1, 0) == _abi.SALT_ERR_INVALID
    assert lib.salt_chi2(None, None, None, None) == _abi.SALT_ERR_INVALID
    assert lib.salt_serve_submit(None, None, None) == _abi.SALT_ERR_INVALID
    h = C.c_void_p()
    assert lib.salt_init_model(None, None, 0, 0, 0, C.byref(h)) == _abi.SALT_ERR_INVALID
    st = _abi.ReplayStats()
    assert _abi.client().salt_client_replay(None, None, 0, None, None, None, None, C.byref(st)) == \
        _abi.SALT_ERR_INVALID
    ps = _abi.PlainStats()
    assert _abi.client().salt_client_plain(None, None, 0, 1.0, 0, None, C.byref(ps)) == _abi.SALT_ERR_INVALID
