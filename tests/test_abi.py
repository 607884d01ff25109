"""The C-ABI library without a GPU: it loads, exports every function
include/emst.h declares, and rejects bad arguments before touching a device."""
import ctypes

import pytest

import paper_2207_00514_gb300 as pkg


@pytest.fixture(scope="module")
def lib():
    from paper_2207_00514_gb300 import _build
    _build.build()
    return pkg.load_library()


def test_exports_every_declared_function(lib):
    names = pkg.declared_functions()
    assert {"emst_compute", "emst_compute_ex", "emst_compute_batched", "emst_status_string",
            "emst_build_bvh", "emst_round_step", "emst_dendrogram"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(lib):
    assert pkg.emst_status_string(0) == "ok"
    for code in range(-7, 0):
        s = pkg.emst_status_string(code)
        assert s and s != "unknown status"
    assert pkg.emst_status_string(42) == "unknown status"


def test_argument_checks_without_gpu(lib):
    V = ctypes.c_void_p
    dummy = ctypes.create_string_buffer(64)
    assert lib.emst_compute(dummy, -1, 3, dummy, V(0)) == -1
    assert lib.emst_compute(dummy, 10, 4, dummy, V(0)) == -1
    assert lib.emst_compute(dummy, 10, 1, dummy, V(0)) == -1
    assert lib.emst_compute(V(0), 10, 3, dummy, V(0)) == -1
    assert lib.emst_compute(dummy, pkg.EMST_MAX_POINTS + 1, 3, dummy, V(0)) == -1
    assert lib.emst_compute(V(0), 0, 3, V(0), V(0)) == 0  # empty input: no work, no device
    I64 = ctypes.c_int64
    assert lib.emst_dendrogram(V(0), I64(-1), V(0), V(0), V(0)) == -1
    assert lib.emst_dendrogram(V(0), I64(pkg.EMST_MAX_POINTS + 1), V(0), V(0), V(0)) == -1
    assert lib.emst_dendrogram(V(0), I64(5), V(0), V(0), V(0)) == -1  # edges missing
    assert lib.emst_dendrogram(V(0), I64(0), V(0), V(0), V(0)) == 0  # nothing to merge


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(pkg.EmstLibraryError):
        pkg.load_library(str(tmp_path / "missing.so"))


def test_oracle_is_not_imported_by_the_product():
    import pathlib
    root = pathlib.Path(pkg.__file__).parent
    for f in list(root.rglob("*.py")) + list(root.rglob("*.cu")) + list(root.rglob("*.cuh")):
        txt = f.read_text()
        assert "import oracle" not in txt and "from oracle" not in txt and "emst_oracle" not in txt, f


def test_dendrogram_binding_rejects_bad_shapes_without_gpu():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        pkg.emst_dendrogram(torch.zeros((5, 2), dtype=torch.int32))      # not (m, 3)
    with pytest.raises(ValueError):
        pkg.emst_dendrogram(torch.zeros((5, 3), dtype=torch.int64))      # not int32
    with pytest.raises(ValueError):
        pkg.emst_dendrogram(torch.zeros((5, 3), dtype=torch.int32), n=9)  # a tree of 9 points has 8 edges
    with pytest.raises(ValueError):
        pkg.emst_dendrogram(torch.zeros((3, 3), dtype=torch.int32),
                            out_linkage=torch.zeros((3, 3), dtype=torch.int32))
    assert pkg.LINKAGE_DTYPE.itemsize == 16
