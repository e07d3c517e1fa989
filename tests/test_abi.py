"""The C ABI library builds, loads, and exports every entry point that
include/*.h declares (CPU only: no device calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("snlm_") and name not in names:
                names.append(name)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1407_2343_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("snlm_denoise", "snlm_patch_dist_1d", "snlm_default_h", "snlm_workspace_bytes",
                     "snlm_status_str", "snlm_nlm_1d", "snlm_denoise_ws", "snlm_denoise_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_python_binding_covers_the_abi():
    from paper_1407_2343_gb300 import _lib, api

    for n in declared_functions():
        assert n in _lib.EXPORTED, n
        assert hasattr(api, n), n


def test_exports_are_c_symbols(lib):
    # plain C names, resolvable through dlsym without C++ mangling
    for n in declared_functions():
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_host_only_entry_points(lib):
    from paper_1407_2343_gb300 import api

    assert api.snlm_default_h(20.0, 3) == pytest.approx(20.0 * 7 ** 0.5, rel=1e-6)
    assert api.snlm_default_h(1.0, 3, "gauss", 2.0) == pytest.approx(2.1509, rel=1e-3)
    assert api.snlm_default_h(-1.0, 3) == -1.0
    assert api.snlm_workspace_bytes(256, 256, "RC") >= 256 * 256 * 4
    assert api.snlm_workspace_bytes(256, 256, "SURE") > api.snlm_workspace_bytes(256, 256, "AVG")
    assert api.snlm_workspace_bytes(0, 256, "RC") == 0
    assert "SNLM_ERR_ARG" in api.snlm_status_str(-1)
    assert api.snlm_version() >= 100


def test_product_path_has_no_oracle_or_fallback():
    # the package never imports the oracle, and has no CPU compute path
    pkg = os.path.join(ROOT, "paper_1407_2343_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "import oracle" not in src and "from oracle" not in src, path
    for path in glob.glob(os.path.join(pkg, "csrc", "*")):
        assert "snlm_oracle" not in open(path).read(), path


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1407_2343_gb300 import _lib

    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(_lib.LibraryMissing):
        _lib.load()


def test_kernel_count_constant_matches_the_binding():
    """SNLM_KERNEL_COUNT (what snlm_preload reports when every kernel loaded) is the
    binding's KERNEL_COUNT, and equals the kernels the preload lists name: 14 pass and
    distance variants and 6 TMA pass variants for each K in 0..7, the batch class
    kernels (6 pass variants for each K in 1..7, and one for the solve and
    combination jobs), 3 recursive-profile modes, 8 SURE kernels, 8 bilateral radii,
    8 2-D NLM half-widths and 4 kernels of the 3-D extension."""
    from paper_1407_2343_gb300 import api

    text = open(os.path.join(ROOT, "include", "snlm.h")).read()
    m = re.search(r"#define\s+SNLM_KERNEL_COUNT\s+(\d+)", text)
    assert m and int(m.group(1)) == api.KERNEL_COUNT
    assert api.KERNEL_COUNT == 8 * (14 + 6) + (7 * 6 + 1) + 3 + 8 + 8 + 8 + 4
