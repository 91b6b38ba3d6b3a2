"""CPU checks of the C-ABI boundary: the library builds, loads, exports every
function declared in include/srt3d.h, and refuses to run without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2203_00952_gb300 import binding
from paper_2203_00952_gb300 import build as builder

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "srt3d.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(srt3d_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    builder.build()
    return binding.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("srt3d_sketch_stream", "srt3d_sketch_hist", "srt3d_reconstruct", "srt3d_submit",
                     "srt3d_poll", "srt3d_create", "srt3d_destroy", "srt3d_finalize", "srt3d_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [name for name in _declared_functions() if not hasattr(lib, name)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(_declared_functions()) <= set(binding._SIGS)


def test_params_struct_layout_matches_header():
    # 5 x 32-bit integers, 6 floats, two 32-bit integers, no padding
    assert ctypes.sizeof(binding.srt3d_params) == 52
    assert binding.srt3d_params.apss_h.offset == 20
    assert binding.srt3d_params.min_sep.offset == 40
    assert binding.srt3d_params.weighting.offset == 44
    assert binding.srt3d_params.birth_every.offset == 48


def test_struct_layouts_against_a_c_compiler(tmp_path):
    # the header compiled by gcc: sizes and offsets of every ABI struct field
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"srt3d_params": binding.srt3d_params, "srt3d_frame": binding.srt3d_frame,
               "srt3d_plan_info": binding.srt3d_plan_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)


def test_frame_struct_layout_matches_header():
    # 3 x 8-byte fields, 4 x uint32, 7 pointers
    assert ctypes.sizeof(binding.srt3d_frame) == 96
    assert binding.srt3d_frame.h.offset == 40


def test_status_strings(lib):
    assert binding.lib().srt3d_status_string(binding.SRT3D_ERANGE) == b"SRT3D_ERANGE"
    assert binding.lib().srt3d_status_string(12345) == b"SRT3D_UNKNOWN"


def test_no_cpu_fallback_without_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.SRT3DError) as ei:
        binding.srt3d_create(0)
    assert ei.value.status == binding.SRT3D_ECUDA


def test_null_context_rejected(lib):
    assert lib.srt3d_sketch_stream(None, None, None, 0, 0, 16, 4, 0, None, None, None) == binding.SRT3D_EINVAL
    assert lib.srt3d_reconstruct(None, None, None, 1, 1, 16, 4, None, None, None, None, None, None,
                                 None) == binding.SRT3D_EINVAL
    for fn in (lib.srt3d_sketch_stream_tc, lib.srt3d_sketch_stream_tc_fused):
        assert fn(None, None, None, 0, 1, 64, 4, binding.SRT3D_FP16_SPLIT, None, None, None) == binding.SRT3D_EINVAL


def test_plan_info_layout():
    # eight uint32 fields and a uint64, as declared in srt3d.h
    assert ctypes.sizeof(binding.srt3d_plan_info) == 40
    assert binding.srt3d_plan_info.serving_frame_bytes.offset == 32
    assert [f for f, _ in binding.srt3d_plan_info._fields_] == [
        "sketch_m", "sketch_lanes", "init_m", "init_grid_spacing", "init_grid_points", "tile_height", "tiles",
        "reserved", "serving_frame_bytes"]
