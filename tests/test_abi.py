"""The C-ABI library builds, loads and exports every entry point include/etp.h declares (no GPU)."""
import os
import re

import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def libetp():
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp
    return etp.lib()


def _declared(root):
    decls = set()
    for name in os.listdir(os.path.join(root, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(root, "include", name)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            decls |= set(re.findall(r"\b(etp_[a-z0-9_]+)\s*\(", text))
    return decls


def test_every_declared_symbol_is_exported(root, libetp):
    decls = _declared(root)
    assert len(decls) >= 20
    missing = [d for d in sorted(decls) if not hasattr(libetp, d)]
    assert not missing, missing


def test_binding_covers_the_abi(root, libetp):
    from paper_2405_05213_gb300 import etp
    for d in _declared(root):
        assert d in etp._SIGS, f"{d} has no ctypes signature"
        assert hasattr(etp, d) or d in ("etp_last_error",), f"{d} has no Python wrapper"


def test_calls_fail_loudly_without_gpu(libetp):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2405_05213_gb300 import etp
    with pytest.raises(etp.EtpError):
        etp.etp_ctx_create(0)
    assert etp.etp_version().startswith("etp")
