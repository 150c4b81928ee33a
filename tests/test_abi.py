"""Host-side checks of the C ABI (no GPU needed): the library builds and
exports every function include/misa.h declares; the binding's structs match
the header's field lists."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "misa.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(misa_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libmisa():
    from paper_2107_07866_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(libmisa):
    names = _declared_functions()
    assert "misa_create" in names and "misa_step" in names and len(names) >= 18
    missing = [n for n in names if not hasattr(libmisa, n)]
    assert not missing, missing


def test_struct_layouts_match_header():
    from paper_2107_07866_gb300 import misa
    src = open(HEADER).read()
    body = re.search(r"typedef struct misa_params \{(.*?)\} misa_params;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1] if not decl.startswith("const") else decl.split(None, 2)[2]
        for nm in names.split(","):
            fields.append(nm.strip().lstrip("*").strip())
    assert [f for f, _ in misa.Params._fields_] == fields
    st = re.search(r"typedef struct misa_stats \{(.*?)\} misa_stats;", src, re.S).group(1)
    st = re.sub(r"/\*.*?\*/", "", st, flags=re.S)
    sfields = []
    for decl in st.split(";"):
        decl = decl.strip()
        if decl:
            sfields += [n.strip() for n in decl.split(None, 1)[1].split(",")]
    assert [f for f, _ in misa.Stats._fields_] == sfields
    pk = re.search(r"typedef struct misa_peaks \{(.*?)\} misa_peaks;", src, re.S).group(1)
    pfields = [d.strip().split()[-1] for d in pk.split(";") if d.strip()]
    assert [f for f, _ in misa.Peaks._fields_] == pfields


def test_tile_shapes_are_warp_parity_pure(libmisa):
    from paper_2107_07866_gb300 import misa
    shapes = misa.tile_shapes()
    assert shapes
    fp64, fp32 = misa.tile_indices("fp64"), misa.tile_indices("fp32")
    assert 1 in fp64 and 1 in fp32
    for k, (tx, ty, tz) in enumerate(shapes, 1):
        cells = tx * ty * tz
        # FP64: one thread per site; FP32: two sites per thread, z folded in
        # halves; each parity fills whole warps, at most 1024 threads
        assert (k in fp64) == (2 * cells <= 1024 and cells % 32 == 0)
        assert (k in fp32) == (tz % 2 == 0 and cells <= 1024 and (cells // 2) % 32 == 0)
    assert libmisa.misa_tile_valid(0, 0) == 0 and libmisa.misa_tile_valid(0, len(shapes) + 1) == 0
    assert libmisa.misa_tile_valid(7, 1) == 0


def test_create_rejects_bad_parameters_without_a_gpu(libmisa):
    # parameter validation happens before any CUDA call
    from paper_2107_07866_gb300 import misa, synth
    pot = synth.potential(n=64)
    with pytest.raises(misa.MisaError) as e:
        misa.Sim(pot, 4, torch_memory=False)
    assert e.value.code == misa.MISA_EINVAL
    with pytest.raises(misa.MisaError) as e:
        misa.Sim(pot, 8, skin=1.5, torch_memory=False)
    assert e.value.code == misa.MISA_EINVAL


def test_build_covers_every_source():
    # every CUDA translation unit under csrc/ is compiled, every header is a
    # rebuild dependency (a stale library would be loaded otherwise)
    import os
    from paper_2107_07866_gb300 import build
    csrc = os.path.join(build.PKG, "csrc")
    units = {os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith(".cu")}
    heads = {os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith(".cuh")}
    assert units == set(build.SOURCES)
    assert heads <= set(build.DEPS) and units <= set(build.DEPS)
    for src in build.SOURCES:
        cmd = build.compile_command(src, "x.o")
        assert "-gencode=arch=compute_103a,code=sm_103a" in cmd and "-c" in cmd
