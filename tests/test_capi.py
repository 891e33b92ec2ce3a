"""The C ABI library loads, exports every function include/mc.h declares, and
rejects invalid configurations before touching the GPU (runs without one)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2212_02197_gb300 import _build, mc, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return mc.lib()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(mc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_function_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(L, n) is not None


def test_status_strings(L):
    assert L.mc_status_str(0) == b"ok"
    assert b"timed out" in L.mc_status_str(4)


def _bad(model=None, ctrl=None, n=10):
    w = workloads.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], **(model or {}))
    c = dict(w["nmpc"], **(ctrl or {}))
    with pytest.raises(mc.McError) as e:
        mc.MonteCarlo(m, c, n, 1)
    assert e.value.status == mc.MC_EINVAL
    return str(e.value)


@pytest.mark.parametrize("model,ctrl,needle", [
    ({}, {"u_min": 900.0}, "u_min <= u_max"),
    ({}, {"N": 0}, "horizon"),
    ({}, {"N": 65}, "horizon"),
    ({"meas_sd": 0.0}, {}, "measurement noise"),
    ({"Ts": 0.0}, {}, "Ts > 0"),
    ({"n_em": 0}, {}, "n_em"),
    ({"V": -1.0}, {}, "positive"),
    ({"sp_time": [0.0, 10.0, 5.0], "sp_value": [1.0, 2.0, 3.0]}, {}, "increase"),
    ({}, {"sqp_tol": 0.0}, "sqp_tol"),
    ({}, {"qp_solver": "ipm", "ip_max_it": 0}, "interior-point"),
    ({}, {"ls_spec_lanes": 33}, "ls_spec_lanes"),
])
def test_invalid_configurations_are_rejected(L, model, ctrl, needle):
    assert needle in _bad(model, ctrl)


def test_negative_size_is_rejected(L):
    assert "n_sims" in _bad(n=-1)


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(mc, "_lib", None)
    monkeypatch.setattr(mc._build, "LIB", "/nonexistent/libmc_gb300.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mc.lib()


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every field of the Python mirrors sits at the offset the C compiler
    gives it in include/mc.h, and the struct sizes agree."""
    import ctypes
    import shutil
    import subprocess

    from paper_2212_02197_gb300 import mc

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    header = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "include", "mc.h")
    structs = {"mc_model_t": mc.McModel, "mc_controller_t": mc.McController,
               "mc_stats_t": mc.McStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{header}"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.splitlines():
        cname, field, value = line.split()
        py = structs[cname]
        if field == "size":
            assert ctypes.sizeof(py) == int(value), cname
        else:
            assert getattr(py, field).offset == int(value), (cname, field)


def test_reduce_noalloc_binding_rejects_bad_arrays_without_a_launch():
    """The binding checks kind, dtype, layout and size of the device arrays
    before it calls the library: nothing here reaches a GPU."""
    import torch

    from paper_2212_02197_gb300 import mc

    phi = torch.zeros(8, dtype=torch.float64)
    cnt = torch.zeros((8, mc.N_COUNTERS), dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA"):
        mc.reduce_noalloc(phi, cnt, 8)
    with pytest.raises(ValueError, match="CUDA torch tensor"):
        mc.reduce_noalloc(123456, cnt, 8)
    with pytest.raises(ValueError):
        mc.reduce_noalloc(phi, cnt, -1)


def test_warp_trace_layout_and_null_arguments(L):
    """The record width is the same in the header, the kernel and the binding,
    and null arguments are rejected before anything touches the device."""
    hdr = open(os.path.join(ROOT, "include", "mc.h")).read()
    assert int(re.search(r"#define MC_WARP_TRACE_WORDS (\d+)", hdr).group(1)) == mc.WARP_TRACE_WORDS
    src = open(os.path.join(ROOT, "paper_2212_02197_gb300", "csrc", "mc_closedloop.cuh")).read()
    assert int(re.search(r"kWarpTraceWords = (\d+)", src).group(1)) == mc.WARP_TRACE_WORDS
    nw = C.c_int64(7)
    assert L.mc_copy_warp_trace(None, None, 0, C.byref(nw)) == mc.MC_EINVAL


def test_new_handle_calls_reject_a_null_handle(L):
    """The gradient's record budget and the per-warp record reject a null
    handle before touching the device."""
    assert L.mc_set_grad_record_budget(None, 0) == mc.MC_EINVAL
    nw = C.c_int64(0)
    assert L.mc_copy_warp_trace(None, None, 0, C.byref(nw)) == mc.MC_EINVAL
    assert L.mc_copy_warp_trace(None, None, -1, C.byref(nw)) == mc.MC_EINVAL
