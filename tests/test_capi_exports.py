"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/phipm.h declares.  No compute call needs a GPU here."""
import ctypes

import pytest

from paper_0907_4631_gb300 import phipm as pm


def _has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_library_builds_and_exports_header_symbols():
    L = pm.lib()
    names = pm.header_functions()
    assert {"phipm_create", "phipm_solve", "phipm_solve_host", "phipm_solve_batched", "phipm_destroy",
            "phipm_last_error", "phipm_default_params", "phipm_set_params"} <= set(names)
    for name in names:
        assert hasattr(L, name), name


def test_default_params_are_the_papers():
    p = pm.default_params()
    assert p.gamma == 0.8 and p.delta == 1.2 and p.m_init == 10 and p.m_max == 64
    assert p.theta13 == 5.37 and p.breakdown_tol == 1e-12 and p.precision == pm.F64


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof / offsetof of every ABI struct, from the C compiler, equal the ctypes mirror."""
    import os
    import subprocess
    structs = {"phipm_csr": pm.CsrC, "phipm_stencil": pm.StencilC, "phipm_function": pm.FunctionC,
               "phipm_operator": pm.OperatorC,
               "phipm_stats": pm.StatsC, "phipm_params": pm.ParamsC, "phipm_trace_record": pm.TraceRecordC,
               "phipm_tune_entry": pm.TuneEntryC}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "phipm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0; }")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


@pytest.mark.skipif(_has_gpu(), reason="checks the no-GPU error path")
def test_create_without_gpu_fails_loudly():
    L = pm.lib()
    h = ctypes.c_void_p()
    st = L.phipm_create(ctypes.byref(h), None)
    assert st == pm.ECUDA and not h.value


def test_invalid_params_rejected_without_gpu():
    L = pm.lib()
    p = pm.default_params()
    p.m_max = 65
    h = ctypes.c_void_p()
    assert L.phipm_create(ctypes.byref(h), ctypes.byref(p)) == pm.EINVAL
    assert not h.value
    p = pm.default_params()
    p.controller = pm.CTRL_LEARNED_STEPS + 1
    assert L.phipm_create(ctypes.byref(h), ctypes.byref(p)) == pm.EINVAL
    assert not h.value
    for bad in (-1, 3):
        p = pm.default_params()
        p.expm_action = bad
        assert L.phipm_create(ctypes.byref(h), ctypes.byref(p)) == pm.EINVAL
        assert not h.value


def test_tuning_entry_points_reject_null_handles(tmp_path):
    """Host-side argument checks of the autotuner's cache calls (no GPU needed)."""
    L = pm.lib()
    path = str(tmp_path / "tune.json").encode()
    assert L.phipm_tune_save(None, path) == pm.EINVAL
    assert L.phipm_tune_load(None, path) == pm.EINVAL
    assert L.phipm_set_team(None, 4) == pm.EINVAL
    assert L.phipm_team_for(None, pm.F64, 0, 1000) == 0


def test_source_hash_ignores_comments_only():
    """The build hash keys stored profiler counters to kernel code: a comment edit must
    leave it unchanged, a code edit must change it, and string literals stay intact."""
    from paper_0907_4631_gb300 import build
    base = 'int f(int a) {\n  return a + 1;  // one\n}\nconst char* s = "a // b";\n'
    assert build._code_only(base) == build._code_only(base.replace("// one", "/* two\n */"))
    assert build._code_only(base) != build._code_only(base.replace("a + 1", "a + 2"))
    assert '"a // b"' in build._code_only(base)
    assert len(build.source_hash()) == 16
