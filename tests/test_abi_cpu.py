"""CPU checks of the C ABI boundary: the in-tree library builds, loads, exports every function
declared in include/sdft.h, and the ctypes structures match the C layouts (gcc, no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdft.h")


@pytest.fixture(scope="module")
def built():
    from paper_2005_10431_gb300 import build
    return build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdft_[a-z0-9_]+)\s*\(", text)) - {"sdft_alloc_fn", "sdft_free_fn"})


def test_library_exports_every_declared_symbol(built):
    names = declared_functions()
    assert len(names) >= 25
    lib = ctypes.CDLL(built)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2005_10431_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == names


def test_ctypes_struct_layouts_match_c(tmp_path):
    from paper_2005_10431_gb300 import _lib
    structs = ["sdft_cell", "sdft_grid", "sdft_atoms", "sdft_pseudo", "sdft_options", "sdft_iter_record",
               "sdft_result"]
    src = tmp_path / "sz.c"
    body = "".join(f'printf("%zu\\n", sizeof({s}));' for s in structs)
    body += 'printf("%zu\\n", offsetof(sdft_options, seed));printf("%zu\\n", offsetof(sdft_options, kT));'
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sdft.h"\nint main(void){' + body + "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    py = [ctypes.sizeof(getattr(_lib, s)) for s in structs]
    py += [_lib.sdft_options.seed.offset, _lib.sdft_options.kT.offset]
    assert out == py


def test_default_options_without_gpu(built):
    import paper_2005_10431_gb300 as sd
    o = sd.sdft_default_options()
    assert (o.nspin, o.nkpt, o.cheb_degree, o.mix_hist, o.precision) == (1, 1, 12, 7, sd.SDFT_FP64)
    assert abs(o.kT - 0.01) < 1e-15 and abs(o.mix_beta - 0.3) < 1e-15
