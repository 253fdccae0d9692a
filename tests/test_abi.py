"""Host-side checks of the boundary: the library builds, loads without a GPU,
exports every function include/bpm.h declares, and the ctypes structs match
the C layout; the input generators are deterministic and conforming."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bpm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1603_09493_gb300 import build
    build.build()
    return L.load()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bpm_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_function_is_exported_and_bound(lib):
    names = _declared()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in L.PROTOTYPES, nm
    assert lib.bpm_version().decode().startswith("bpmllg")


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "bpm.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(bpm_island), sizeof(bpm_run_params),'
                   ' sizeof(bpm_region_mat), sizeof(bpm_mesh_info), offsetof(bpm_run_params, map_id),'
                   ' offsetof(bpm_island, Hext_T));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(L.bpm_island), ctypes.sizeof(L.bpm_run_params),
                   ctypes.sizeof(L.bpm_region_mat), ctypes.sizeof(L.bpm_mesh_info),
                   L.bpm_run_params.map_id.offset, L.bpm_island.Hext_T.offset]
    assert L.ISLAND_DTYPE.itemsize == ctypes.sizeof(L.bpm_island) == 44


def test_every_struct_matches_its_ctypes_twin(tmp_path):
    # every field offset and every size, for each header struct the binding mirrors
    structs = [getattr(L, n) for n in dir(L) if n.startswith("bpm_") and isinstance(getattr(L, n), type)
               and issubclass(getattr(L, n), ctypes.Structure)]
    assert len(structs) >= 8
    lines, want = [], []
    for st in structs:
        lines.append(f'printf("%zu\\n", sizeof({st.__name__}));')
        want.append(ctypes.sizeof(st))
        for fname, _ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st.__name__}, {fname}));')
            want.append(getattr(st, fname).offset)
    src = tmp_path / "layout.c"
    src.write_text('#include "bpm.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){\n' +
                   "\n".join(lines) + "\nreturn 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-pedantic", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == want


def test_a_c_program_links_every_declared_function(lib, tmp_path):
    # the declarations, compiled as C99, resolve against the built library
    names = _declared()
    src = tmp_path / "link.c"
    src.write_text('#include "bpm.h"\n#include <stdio.h>\nint main(void){\n' +
                   "\n".join(f'printf("%p\\n", (void*){n});' for n in names) + "\nreturn 0;}\n")
    exe = tmp_path / "link"
    libdir = os.path.dirname(L.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-pedantic", "-Wall", "-Werror", "-Wno-pedantic",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lbpmllg",
                           f"-Wl,-rpath,{libdir}"])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and len(out.stdout.split()) == len(names)


def test_no_gpu_calls_fail_cleanly(lib):
    # without a GPU the library reports an error instead of crashing
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.bpm_create(ctypes.byref(h), 0, None)
    assert rc in (-1, -2)
    assert lib.bpm_last_error().decode() != ""


def test_counter_rng_is_reproducible_per_index():
    a = synth.counter_normal(7, 3, np.arange(100, dtype=np.uint64))
    b = synth.counter_normal(7, 3, np.arange(50, 100, dtype=np.uint64))
    assert np.array_equal(a[50:], b)
    assert abs(a.mean()) < 0.3 and 0.7 < a.std() < 1.3
    j1 = synth.jittered_islands(10, seed=1)
    j2 = synth.jittered_islands(4, seed=1, first_index=6)
    assert np.array_equal(j1.Ms_scale[6:], j2.Ms_scale)


@pytest.mark.parametrize("maker", [synth.small_island_mesh, synth.census_island_mesh,
                                   lambda: synth.variant_island_mesh(10.0, 0.4, True, 3000, 5)])
def test_meshes_are_conforming(maker):
    m = maker()
    faces = np.sort(np.concatenate([m.tets[:, [1, 2, 3]], m.tets[:, [0, 2, 3]], m.tets[:, [0, 1, 3]],
                                    m.tets[:, [0, 1, 2]]]), axis=1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert counts.max() == 2
    # boundary faces = two end caps + lateral quads (2 triangles each)
    K = m.info["rings"]
    slabs = m.info["planes"] - 1
    assert (counts == 1).sum() == 2 * 6 * K * K + 2 * 6 * K * slabs
