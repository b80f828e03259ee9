"""The C-ABI library loads and exports every entry point include/*.h
declares, and its host-only calls behave (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__
from paper_2606_24531_gb300 import ace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ace_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported_and_bound():
    declared = _declared()
    assert {"ace_index_build", "ace_decode_all", "ace_seek", "ace_verify"} <= declared
    lib = ace.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", ace._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ace_[a-z0-9_]+)", out))
    assert declared <= exported, declared - exported
    assert declared <= set(ace.exported_symbols()), declared - set(ace.exported_symbols())
    for name in declared:
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_names():
    names = [ace.ace_status_str(i) for i in range(7)]
    assert names == ["ACE_OK", "ACE_E_INVAL", "ACE_E_CORRUPT", "ACE_E_RANGE", "ACE_E_NOMEM",
                     "ACE_E_TIMEOUT", "ACE_E_CUDA"]


def test_index_size_reads_the_header_on_the_host():
    data = np.frombuffer(b"hello hello hello hello world" * 100, np.uint8)
    arc = ace.ace_encode(data, 8, 4)
    nb = (data.size + 255) // 256
    size = ace.ace_index_size(arc[:64])
    assert size >= 256 + 4 * nb
    bad = arc[:64].copy()
    bad[0] ^= 1  # magic
    with pytest.raises(ace.AceError) as e:
        ace.ace_index_size(bad)
    assert e.value.status == ace.ACE_E_CORRUPT
    bad = arc[:64].copy()
    bad[24] ^= 1  # n_blocks no longer matches total_size
    with pytest.raises(ace.AceError):
        ace.ace_index_size(bad)


def test_encode_bound_and_params():
    assert ace.ace_encode_bound(0, 14) > 0
    assert ace.ace_encode_bound(1 << 20, 14) > (1 << 20)
    with pytest.raises(ace.AceError):
        ace.ace_encode(np.zeros(10, np.uint8), 7, 4)   # block too small
    with pytest.raises(ace.AceError):
        ace.ace_encode(np.zeros(10, np.uint8), 14, 3)  # min match below 4
