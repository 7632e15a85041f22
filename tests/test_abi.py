"""The C-ABI library builds, loads without a GPU, and exports every function
that include/cutqc.h declares.  No compute calls here."""
import ctypes
import subprocess

import pytest


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc
    return cutqc


def test_exports_every_declared_symbol(built):
    cutqc = built
    declared = cutqc.declared_symbols()
    assert len(declared) >= 12
    L = cutqc.lib()
    for name in declared:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", cutqc.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(declared) <= exported


def test_version_and_error_text(built):
    cutqc = built
    assert "sm_103a" in cutqc.cutqc_version()
    assert isinstance(cutqc.cutqc_last_error(), str)


def test_host_validation_without_gpu(built):
    """Descriptor checks run on the host before any CUDA call."""
    cutqc = built

    class S:
        w = 3
        in_local = [2, 1]          # not ascending: rejected
        out_local = []
        in_edge = [0, 1]
        out_edge = []
        out_qubit = [0, 1, 2]
    with pytest.raises(cutqc.CutqcError) as e:
        cutqc.cutqc_attribute_workspace_size(S)
    assert e.value.code == cutqc.EINVAL

    class T:
        w = 4
        in_local = [0]
        out_local = [3]
        in_edge = [0]
        out_edge = [1]
        out_qubit = [0, 1, 2]
    assert cutqc.cutqc_attribute_workspace_size(T) == 4 * 3 * 16 * 4

    class U:
        w = 3
        in_local = []
        out_local = [2]
        in_edge = []
        out_edge = [0]
        out_qubit = [0, 1]

    class V:
        w = 3
        in_local = [0]
        out_local = []
        in_edge = [0]
        out_edge = []
        out_qubit = [2, 3, 4]
    assert cutqc.cutqc_fd_shape([U, V]) == (4, 8)
    with pytest.raises(cutqc.CutqcError):      # edge 0 measured twice
        cutqc.cutqc_fd_shape([U, U])
