"""The C ABI from C: include/lp.h compiles as strict C99 and C++17, a C program links against the
built library and calls its host-only entry points, and every struct has the size and field
offsets the Python binding assumes (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "lp_params": ["tol", "cg_rel_tol", "sigma", "gamma", "cg_max_iter", "ipm_max_iter",
                  "refine_max", "sketch_s", "sketch_w", "cg_theory_rule", "seed", "stream_dtype",
                  "cg_batch", "inner_solver", "sketch_kind", "use_graphs",
                  "gram_tensor_cores", "autotune", "shared_cg", "persistent_cg", "factor_dag"],
    "lp_info": ["ipm_iters", "cg_iters_total", "cg_iters_last", "refine_steps", "rp_rel",
                "rd_rel", "gap_rel", "mu", "obj", "alpha_max", "alpha", "f_norm", "v_norm",
                "status", "f_target", "stream_dtype", "stream_switch_iter", "factor_two_stage",
                "cg_precise_iter", "cg_graph_solves", "cg_persistent_solves"],
    "lp_ipm_state": ["k", "stream_switch_iter", "r0", "mu0"],
    "lp_profile": ["phase_ms", "phase_calls", "matvec_ms", "matvec_count", "matvec_bytes",
                   "launches", "tune_tc", "tune_stages", "tune_ctas", "tune_us", "tune_rule_us"],
}


@pytest.fixture(scope="module")
def libpath():
    from paper_2003_08072_gb300 import build

    return build.build()


def _c_source():
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include \"lp.h\"", "int main(void) {"]
    for st, fields in STRUCTS.items():
        lines.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'  printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    for name in ("lp_profile", "lp_server_stats_t"):
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
    lines += [
        "  lp_params p;",
        "  if (lp_params_default(&p) != LP_OK) return 2;",
        '  printf("default tol %.3g sigma %.3g s %d\\n", p.tol, p.sigma, (int)p.sketch_s);',
        '  printf("status %s\\n", lp_status_str(LP_ERR_BREAKDOWN));',
        "  if (lp_params_default(NULL) != LP_ERR_ARG) return 3;",
        "  return 0;",
        "}",
    ]
    return "\n".join(lines) + "\n"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_header_is_c99_and_layouts_match_the_binding(tmp_path, libpath):
    from paper_2003_08072_gb300 import _binding as B

    src = tmp_path / "abi.c"
    src.write_text(_c_source())
    exe = tmp_path / "abi"
    libdir = os.path.dirname(libpath)
    lib = os.path.basename(libpath)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-l:" + lib, "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.splitlines() if not line.startswith(("default", "status")))
    for st, fields in STRUCTS.items():
        cls = getattr(B, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fields:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
    for name in ("lp_profile", "lp_server_stats_t"):
        assert int(got[name]) == ctypes.sizeof(getattr(B, name)), name
    assert "default tol 1e-08 sigma 0.5 s 4" in out
    assert "status LP_ERR_BREAKDOWN" in out


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_header_compiles_as_cpp(tmp_path):
    src = tmp_path / "abi.cpp"
    src.write_text("#include \"lp.h\"\nint main() { lp_params p; return lp_params_default(&p); }\n")
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                    "-I", os.path.join(ROOT, "include"), str(src)], check=True)
