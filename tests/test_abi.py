"""C-ABI checks that need no GPU: the library loads, exports every function
include/accsink.h declares, and the ctypes structs match the C layouts."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "accsink.h")


@pytest.fixture(scope="module")
def L():
    from paper_2605_30267_gb300 import build
    build.build()
    from paper_2605_30267_gb300 import binding
    return binding.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(accsink_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("accsink_create", "accsink_destroy", "accsink_solve", "accsink_solve_host",
                 "accsink_row_pass", "accsink_col_lse", "accsink_sinkhorn_map",
                 "accsink_transport_cost", "accsink_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    from paper_2605_30267_gb300 import binding
    names = declared_functions()
    for name in names:
        assert hasattr(L, name), f"{name} declared in accsink.h but not exported"
    assert sorted(binding.EXPORTED) == names
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(accsink_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_c(tmp_path):
    """Compile a C program against the header and compare sizeof/offsetof."""
    from paper_2605_30267_gb300 import binding as B
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "accsink.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(accsink_problem), offsetof(accsink_problem, ldc),
         offsetof(accsink_problem, a), offsetof(accsink_problem, cost_scale),
         offsetof(accsink_problem, b));
  printf("%zu %zu %zu %zu\n", sizeof(accsink_params), offsetof(accsink_params, eps),
         offsetof(accsink_params, max_sinkhorn_steps), offsetof(accsink_params, history));
  printf("%zu %zu %zu\n", sizeof(accsink_result), offsetof(accsink_result, marginal_l1),
         offsetof(accsink_result, gpu_ms));
  printf("%zu %zu %zu %zu\n", sizeof(accsink_batch_config),
         offsetof(accsink_batch_config, row_tile_elems), offsetof(accsink_batch_config, ctas_per_sm),
         offsetof(accsink_batch_config, dense_solo_min_nm));
  printf("%zu %zu %zu\n", sizeof(accsink_server_stats),
         offsetof(accsink_server_stats, resident_bytes), offsetof(accsink_server_stats, busy_ms));
  printf("%zu %zu %zu %zu %zu\n", sizeof(accsink_state), offsetof(accsink_state, eps),
         offsetof(accsink_state, eps_c), offsetof(accsink_state, x), offsetof(accsink_state, w));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    p = [int(v) for v in lines[0].split()]
    assert p == [ct.sizeof(B.accsink_problem), B.accsink_problem.ldc.offset,
                 B.accsink_problem.a.offset, B.accsink_problem.cost_scale.offset,
                 B.accsink_problem.b.offset]
    q = [int(v) for v in lines[1].split()]
    assert q == [ct.sizeof(B.accsink_params), B.accsink_params.eps.offset,
                 B.accsink_params.max_sinkhorn_steps.offset, B.accsink_params.history.offset]
    r = [int(v) for v in lines[2].split()]
    assert r == [ct.sizeof(B.accsink_result), B.accsink_result.marginal_l1.offset,
                 B.accsink_result.gpu_ms.offset]
    c = [int(v) for v in lines[3].split()]
    assert c == [ct.sizeof(B.accsink_batch_config), B.accsink_batch_config.row_tile_elems.offset,
                 B.accsink_batch_config.ctas_per_sm.offset,
                 B.accsink_batch_config.dense_solo_min_nm.offset]
    v = [int(x) for x in lines[4].split()]
    assert v == [ct.sizeof(B.accsink_server_stats), B.accsink_server_stats.resident_bytes.offset,
                 B.accsink_server_stats.busy_ms.offset]
    t = [int(x) for x in lines[5].split()]
    assert t == [ct.sizeof(B.accsink_state), B.accsink_state.eps.offset,
                 B.accsink_state.eps_c.offset, B.accsink_state.x.offset, B.accsink_state.w.offset]


def test_host_only_calls(L):
    from paper_2605_30267_gb300 import binding as B
    p = B.default_params()
    assert p.method == B.ACC and p.eps == 1e-2 and p.tol == 1e-6 and p.mu0 == 0.25
    assert p.m0 == 4 and p.carry == B.CARRY_Y and p.use_graph == 1
    assert L.accsink_version().decode().startswith("accsink")
    assert L.accsink_last_error(None).decode() == "NULL context"


def test_build_targets_sm103a_only():
    from paper_2605_30267_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2605_30267_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "acc_sinkhorn_oracle" not in text, f
