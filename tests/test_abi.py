"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares
(no compute call: this runs without a GPU)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(tucker_[a-z_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2308_16395_gb300 import build as b

    path = b.build()
    import paper_2308_16395_gb300 as pkg

    return pkg.load_library(), path


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tucker_init_sthosvd", "tucker_stream_update", "tucker_reconstruct",
                     "tucker_error_norm"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    _, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tucker_[a-z_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(lib):
    import paper_2308_16395_gb300 as pkg

    for n in _declared():
        assert hasattr(pkg, n), n
    assert set(pkg.EXPORTS) == set(_declared())


def test_library_is_built_for_sm_103a():
    """The build compiles every translation unit for sm_103a and nothing else."""
    from paper_2308_16395_gb300 import build as b

    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert all(f not in b._flags() for f in ("-arch=native", "-march=native"))


def test_config_struct_size_matches_header(lib):
    import ctypes

    import paper_2308_16395_gb300 as pkg

    # 4 int32 + 8 int64 + 8 int64 + 2 int64 + 2 double
    assert ctypes.sizeof(pkg.TuckerConfig) == 16 + 64 + 64 + 16 + 16


def test_version_string(lib):
    import paper_2308_16395_gb300 as pkg

    assert "sm_103a" in pkg.tucker_version()


def test_ttm_workspace_query_is_host_only(lib):
    """tucker_ttm_workspace_bytes: 4 buffers of max_k N r_k / n_k elements, 256-byte rounded;
    -1 for an invalid descriptor (no device call)."""
    import paper_2308_16395_gb300 as pkg

    d = pkg.ttm_desc((128, 128, 64), (20, 20, 12), "f32")
    M = max(128 * 128 * 64 // n * r for n, r in zip((128, 128, 64), (20, 20, 12)))
    assert pkg.tucker_ttm_workspace_bytes(d) == 4 * ((M * 4 + 255) // 256 * 256)
    for n, r in [((8, 8), (9, 2)), ((8, 0), (2, 0)), ((), ())]:
        with pytest.raises(pkg.TuckerError):
            pkg.tucker_ttm_workspace_bytes(pkg.ttm_desc(n, r, "f64"))


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the C compiler's size and field offsets (the header
    compiled as C by gcc; no GPU and no CUDA library needed)."""
    import ctypes
    import shutil

    import paper_2308_16395_gb300 as pkg

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("tucker_config", pkg.TuckerConfig), ("tucker_step_info", pkg.StepInfo),
             ("tucker_profile", pkg.Profile), ("tucker_launch_plan", pkg.LaunchPlan),
             ("tucker_ttm_desc", pkg.TtmDesc), ("tucker_step_record", pkg.StepRecord),
             ("tucker_replay", pkg.Replay), ("tucker_recompress_info", pkg.RecompressInfo)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tucker_stream.h"',
             '#include "tucker_ttm.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
