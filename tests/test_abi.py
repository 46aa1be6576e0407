"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports
every entry point include/vbm.h declares, validates arguments on the host, and its FP64
host bank agrees with the oracle's."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_09417_gb300 import build_ext, vbm
    build_ext.build()
    return vbm


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names.update(re.findall(r"VBM_API[^;(]*?\b(vbm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    handle = lib.load()
    for n in names:
        assert hasattr(handle, n), n
    assert names == set(lib.EXPORTED)
    assert lib.version() == 101


def test_struct_sizes_match_header(lib):
    assert ctypes.sizeof(lib.Camera) == 80
    assert ctypes.sizeof(lib.TF) == 4 + 16 * 4 + 16 * 16
    assert ctypes.sizeof(lib.BankEntry) == 128


def test_struct_layouts_match_header(lib, tmp_path):
    """Every struct the binding declares has the header's size and, field by field, the
    header's offsets (a C program compiled against include/vbm.h prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = [("vbm_camera", lib.Camera), ("vbm_tf", lib.TF), ("vbm_bank_entry", lib.BankEntry),
               ("vbm_bank", lib.Bank), ("vbm_select", lib.Select), ("vbm_plan_desc", lib.PlanDesc),
               ("vbm_plan_buffers", lib.PlanBuffers)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vbm.h"', "int main(void) {"]
    for cname, cls in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines.append("return 0; }")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines))
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", include, "-o", str(exe), str(src)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, cls in structs:
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert int(got[cname + "." + f[0]]) == getattr(cls, f[0]).offset, (cname, f[0])


def test_host_argument_validation(lib):
    with pytest.raises(lib.VbmError) as e:
        lib.Plan([0, 10], 2, 64, 64, tile_w=16, tile_h=12)      # 192-pixel tiles are not supported
    assert e.value.status == lib.VBM_ERR_ARG
    with pytest.raises(lib.VbmError) as e:
        lib.Plan([0, 10, 5], 2, 64, 64, view_scene=[0, 1])       # decreasing offsets
    assert e.value.status == lib.VBM_ERR_ARG
    with pytest.raises(lib.VbmError) as e:
        lib.Plan([0, 10], 1, 8 * 65536, 64, tile_w=8, tile_h=8)  # 65536 tiles across: the placement
    assert e.value.status == lib.VBM_ERR_ARG                    # record packs tile columns in 16 bits
    assert "65535 tiles" in lib.load().vbm_last_error().decode()
    with pytest.raises(lib.VbmError) as e:
        lib.bank_build(0, 0)
    assert e.value.status == lib.VBM_ERR_ARG
    assert "levels" in lib.load().vbm_last_error().decode()


@pytest.mark.parametrize("levels,wavelet", [(2, 0), (4, 0), (5, 0), (1, 1), (3, 1), (5, 1)])
def test_host_bank_matches_oracle(lib, levels, wavelet):
    """Every entry of the library's bank against the oracle's, up to the five bior4.4
    levels of the 512^3 workload (levels 3 and up take the oracle's separable kernel)."""
    from _helpers import oracle_bank
    got = lib.bank_to_dicts(lib.bank_build(levels, wavelet))
    ref = oracle_bank(levels, wavelet)
    assert len(got) == len(ref) == 7 * levels + 1
    for a, b in zip(got, ref):
        assert (a["j"], tuple(a["o"])) == (b["j"], tuple(b["o"]))
        assert np.allclose(a["u"], b["u"], atol=1e-9)
        assert np.allclose(a["cov"], b["cov"], atol=1e-10)
        assert abs(a["w"] - b["w"]) < 1e-10 * b["w"]
        assert np.allclose(a["log_scale"], b["log_scale"], atol=1e-6)
        assert np.allclose(a["quat"], b["quat"], atol=1e-7)


@pytest.mark.parametrize("wavelet,flags", [(0, 1), (0, 2), (1, 3)])
def test_host_bank_ablation_matches_oracle(lib, wavelet, flags):
    """vbm_bank_ablate (host only) against the oracle's ablation of its own bank."""
    from _helpers import oracle_bank
    bank = lib.bank_build(3, wavelet)
    ref = oracle_bank(3, wavelet, ablation=flags)
    got = lib.bank_to_dicts(lib.bank_ablate(bank, flags))
    for a, b in zip(got, ref):
        assert np.allclose(a["u"], b["u"], atol=1e-9) and np.allclose(a["cov"], b["cov"], rtol=1e-10, atol=1e-10)
        assert abs(a["w"] - b["w"]) <= 1e-10 * abs(b["w"])
        assert np.allclose(a["log_scale"], b["log_scale"], atol=1e-6)
        assert np.allclose(a["quat"], b["quat"], atol=1e-7)
    with pytest.raises(lib.VbmError) as e:
        lib.bank_ablate(lib.bank_build(2, 0), 8)
    assert e.value.status == lib.VBM_ERR_ARG

