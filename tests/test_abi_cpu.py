"""The C-ABI library builds, loads and exports every declared entry point (no GPU work)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1401_7457_gb300 import build, binding
    build.build()
    return binding.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cxbwt_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    from paper_1401_7457_gb300 import binding
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in binding.SIGNATURES, f"{name} has no binding"


def test_abi_version(lib):
    assert lib.cxbwt_abi_version() == 3


def test_pack_unpack_roundtrip(lib):
    from paper_1401_7457_gb300 import binding
    rng = np.random.default_rng(0)
    for n in [0, 1, 15, 16, 17, 1000]:
        codes = rng.integers(0, 4, size=n, dtype=np.uint8)
        w = binding.pack_codes(codes)
        assert w.size == (n + 15) // 16
        s = "".join("ACGT"[c] for c in codes)
        assert np.array_equal(binding.pack_ascii(s), w)
        # unpack with two '$' positions
        if n >= 3:
            got = binding.unpack_ascii(w, np.array([0, n - 1], dtype=np.uint64), n)
            assert got == ("$" + s[1:-1] + "$").encode()
    # bit layout: base j at bits 31-2j .. 30-2j of word 0
    assert binding.pack_ascii("CA")[0] == 1 << 30
    assert binding.pack_ascii("AAAAAAAAAAAAAAAT")[0] == 3


def test_helpers_reject_bad_input(lib):
    from paper_1401_7457_gb300 import binding
    with pytest.raises(binding.CxbwtError):
        binding.pack_ascii("ACGN")
    with pytest.raises(binding.CxbwtError):
        binding.pack_codes(np.array([0, 4], dtype=np.uint8))
    with pytest.raises(binding.CxbwtError):
        binding.unpack_ascii(np.zeros(1, dtype=np.uint32), np.array([20], dtype=np.uint64), 16)


def test_output_size(lib):
    from paper_1401_7457_gb300 import binding
    assert binding.output_size(np.array([4, 4, 4], dtype=np.uint32)) == (15, 1)
    assert binding.output_size(np.array([100] * 10000, dtype=np.uint32)) == (1_010_000, 63_125)


def test_status_strings(lib):
    lib.cxbwt_status_string.restype = ctypes.c_char_p
    assert lib.cxbwt_status_string(-4) == b"CXBWT_ETIMEOUT"


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that the C compiler gives the header's struct (a mismatch would pass
    garbage through the ABI without an error)."""
    import shutil
    import subprocess

    from paper_1401_7457_gb300 import binding
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"cxbwt_options": binding.Options, "cxbwt_stats": binding.Stats, "cxbwt_tuning": binding.Tuning,
               "cxbwt_server_options": binding.ServerOptions, "cxbwt_request": binding.Request,
               "cxbwt_collection": binding.Collection}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "cxbwt.h"', "int main(void) {"]
    want = []
    for cname, py in structs.items():
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            field = getattr(py, fname)
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname.rstrip("_")}));')
            want.append(field.offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want


def test_binding_signatures_match_the_header():
    """Each entry point's ctypes signature takes as many arguments as its C
    prototype, and returns a value exactly when the prototype does."""
    from paper_1401_7457_gb300 import binding
    protos = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for ret, name, params in re.findall(r"([\w\s\*]+?)\b(cxbwt_\w+)\s*\(([^)]*)\)\s*;", text):
                params = params.strip()
                n = 0 if params in ("", "void") else params.count(",") + 1
                protos[name] = (ret.split()[-1] != "void" or "*" in ret, n)
    assert set(protos) == set(binding.SIGNATURES)
    for name, (returns, n) in protos.items():
        restype, argtypes = binding.SIGNATURES[name]
        assert len(argtypes) == n, name
        assert (restype is not None) == returns, name


def test_binding_rejects_wrong_element_sizes():
    """Arrays whose elements the library would misread are refused before
    any call: lengths as int64, packed words as uint8 codes, $ rows as
    uint32."""
    import torch

    from paper_1401_7457_gb300 import binding
    binding._need(4, reads_2bit=np.zeros(3, dtype=np.uint32), lens=torch.zeros(2, dtype=torch.int32), none=None)
    binding._need(8, out_dollar_pos=np.zeros(2, dtype=np.uint64), out_counts=torch.zeros(5, dtype=torch.int64))
    with pytest.raises(TypeError, match="lens needs 4-byte"):
        binding._need(4, lens=np.array([100, 100]))  # numpy's default int64
    with pytest.raises(TypeError, match="reads_2bit needs 4-byte"):
        binding._need(4, reads_2bit=np.zeros(16, dtype=np.uint8))
    with pytest.raises(TypeError, match="out_dollar_pos needs 8-byte"):
        binding._need(8, out_dollar_pos=torch.zeros(2, dtype=torch.int32))


def test_create_rejects_options_it_does_not_build(lib):
    """Checked before any device work, so this runs without a GPU."""
    from paper_1401_7457_gb300 import binding
    for field, value in (("prefix_len", 4), ("prefix_len", 8), ("prefix_len", 20), ("digit_bits", 4)):
        opt = binding.Options()
        lib.cxbwt_default_options(ctypes.byref(opt))
        setattr(opt, field, value)
        h = ctypes.c_void_p()
        assert lib.cxbwt_create(ctypes.byref(h), ctypes.byref(opt)) == -5
        assert not h.value
        assert field.encode() in lib.cxbwt_last_error(None)


def test_no_cpu_fallback(lib, monkeypatch):
    """Without a CUDA device a context cannot be created (CXBWT_ECUDA): the
    library has no CPU path.  Without the built library the binding raises
    instead of computing anything itself."""
    import torch

    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        with pytest.raises(binding.CxbwtError) as e:
            binding.Context(device=0)
        assert e.value.status == -3
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libcxbwt.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.pack_codes(np.zeros(4, dtype=np.uint8))


def test_create_accepts_group_depths_it_builds(lib):
    """prefix_len 0, 12 and 16 pass the option check: without a GPU the call
    then fails for want of a device (CXBWT_ECUDA), not for the option."""
    import torch

    from paper_1401_7457_gb300 import binding
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: creation would succeed")
    for value in (0, 12, 16):
        opt = binding.Options()
        lib.cxbwt_default_options(ctypes.byref(opt))
        opt.prefix_len = value
        h = ctypes.c_void_p()
        assert lib.cxbwt_create(ctypes.byref(h), ctypes.byref(opt)) == -3
        assert b"prefix_len" not in lib.cxbwt_last_error(None)
