"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and exports
every function include/aps.h declares; the product path and the oracle stay separate."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aps.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(aps_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1402_3010_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("aps_build_index", "aps_all_pairs", "aps_query", "aps_stream_submit", "aps_stream_poll",
                     "aps_batch_all_pairs", "aps_all_pairs_dense", "aps_pairs_free", "aps_index_free",
                     "aps_last_error"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a(lib):
    from paper_1402_3010_gb300 import _build

    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    cuobj = shutil.which("cuobjdump") or "/usr/local/cuda/bin/cuobjdump"
    if not os.path.exists(cuobj):
        pytest.skip("cuobjdump not available")
    out = subprocess.run([cuobj, "--list-elf", _build.LIB], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_version_and_error_calls_need_no_gpu(lib):
    lib.aps_version.restype = ctypes.c_char_p
    lib.aps_last_error.restype = ctypes.c_char_p
    assert b"aps" in lib.aps_version()
    assert isinstance(lib.aps_last_error(), bytes)


def _imports(txt):
    return re.findall(r"^\s*(?:import|from)\s+([\w.]+)|^\s*#include\s+[<\"]([^>\"]+)", txt, flags=re.M)


def test_product_and_oracle_share_no_code():
    pkg = os.path.join(ROOT, "paper_1402_3010_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                for a, b in _imports(open(os.path.join(dirpath, f)).read()):
                    mod = a or b
                    assert not mod.startswith("oracle") and "aps_oracle" not in mod, (f, mod)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            for a, b in _imports(open(os.path.join(ROOT, "oracle", f)).read()):
                mod = a or b
                assert not mod.startswith("paper_1402_3010_gb300") and "aps.h" not in mod, (f, mod)


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    import paper_1402_3010_gb300 as aps

    monkeypatch.setattr(aps, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(aps, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        aps.load()


def test_variant_table_matches_header():
    """The binding's VARIANTS table and the APS_VARIANT_* macros name the same flag sets."""
    import paper_1402_3010_gb300 as A

    txt = open(HEADER).read()
    flags = {k: int(v, 16) for k, v in re.findall(r"#define (APS_NO_[A-Z_]+) (0x[0-9a-f]+)u", txt)}
    macros = dict(re.findall(r"#define APS_VARIANT_([A-Z0-9_]+) (.+)", txt))
    got = {}
    for name, expr in macros.items():
        v = 0
        for tok in re.findall(r"APS_NO_[A-Z_]+", expr):
            v |= flags[tok]
        got["all-pairs-" + name[len("ALL_PAIRS_"):].lower().replace("_", "-")] = v
    want = {("all-pairs-0" if k == "all-pairs-0-array" else "all-pairs-1" if k == "all-pairs-1-array" else k): v
            for k, v in A.VARIANTS.items()}
    assert got == want
    assert len(got) == 9


def test_noalloc_binding_rejects_host_and_mistyped_outputs():
    """The allocation-free join's outputs are written by kernels: the binding refuses a
    NumPy array, a CPU tensor, a wrong dtype and a strided view before calling the library
    (no GPU needed; the checks run first)."""
    import numpy as np
    import torch

    import paper_1402_3010_gb300 as aps

    i32 = np.zeros(8, np.int32)
    f32 = np.zeros(8, np.float32)
    with pytest.raises(ValueError):
        aps.aps_all_pairs_noalloc(0, i32, i32, f32)
    ti = torch.zeros(8, dtype=torch.int32)
    tf = torch.zeros(8, dtype=torch.float32)
    with pytest.raises(ValueError):
        aps.aps_all_pairs_noalloc(0, ti, ti, tf)
    if torch.cuda.is_available():  # pragma: no cover - CPU suite
        di = torch.zeros(8, dtype=torch.int16, device="cuda")
        with pytest.raises(ValueError):
            aps.aps_all_pairs_noalloc(0, di, di, di)
