"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/at.h declares, its structs have the layout the
binding assumes, and host-side argument validation rejects bad input."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "at.h")


@pytest.fixture(scope="module")
def B():
    from paper_1911_05769_gb300 import build
    build.build()
    from paper_1911_05769_gb300 import binding
    binding.lib()
    return binding


def _declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(at_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_abi():
    names = _declared_functions()
    for must in ("at_create", "at_step", "at_state", "at_destroy", "at_set_state", "at_workspace_bytes",
                 "at_status", "at_delay_stats", "at_get_info", "at_last_error", "at_create_batch",
                 "at_batch_workspace_bytes", "at_tune"):
        assert must in names


def test_library_exports_every_declared_symbol(B):
    out = subprocess.check_output(["nm", "-D", "--defined-only", B.library_path()], text=True)
    exported = set(re.findall(r"\sT\s+(at_\w+)$", out, flags=re.M))
    declared = set(_declared_functions())
    assert declared <= exported, declared - exported
    assert exported <= declared, exported - declared
    assert set(B.EXPORTED) == declared
    lib = B.lib()
    for name in declared:
        assert getattr(lib, name) is not None


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "at.h"
#define F(S, m) printf(#S " " #m " %zu\n", offsetof(S, m))
int main(void) {
  printf("at_grid size %zu\n", sizeof(at_grid));
  F(at_grid, dim); F(at_grid, bc); F(at_grid, dtype); F(at_grid, flags); F(at_grid, n); F(at_grid, length);
  F(at_grid, origin); F(at_grid, forcing_amp); F(at_grid, seed); F(at_grid, workspace);
  F(at_grid, workspace_bytes); F(at_grid, stream); F(at_grid, timeout_ns); F(at_grid, max_ctas);
  F(at_grid, stages); F(at_grid, test_skip_step); F(at_grid, steps_per_pass); F(at_grid, tile_subdomains);
  F(at_grid, sub);
  printf("at_info size %zu\n", sizeof(at_info));
  F(at_info, N); F(at_info, P); F(at_info, M); F(at_info, order); F(at_info, L); F(at_info, R); F(at_info, s);
  F(at_info, T); F(at_info, ctas); F(at_info, threads); F(at_info, stages); F(at_info, smem_bytes);
  F(at_info, step); F(at_info, sm_count); F(at_info, dtype); F(at_info, steps_per_pass); F(at_info, viscous_fp64);
  F(at_info, tile_subdomains);
  printf("at_instance size %zu\n", sizeof(at_instance));
  F(at_instance, n); F(at_instance, L); F(at_instance, bc); F(at_instance, length); F(at_instance, origin);
  F(at_instance, nu); F(at_instance, dt); F(at_instance, tanh_a); F(at_instance, tanh_c); F(at_instance, tanh_xc);
  F(at_instance, seed);
  printf("at_tune_result size %zu\n", sizeof(at_tune_result));
  F(at_tune_result, ctas); F(at_tune_result, stages); F(at_tune_result, steps_per_pass);
  F(at_tune_result, tile_subdomains);
  F(at_tune_result, n_tried); F(at_tune_result, best_ms); F(at_tune_result, first_ms);
  return 0;
}
"""


def test_struct_layout_matches_binding(B, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    lines = subprocess.check_output([str(exe)], text=True).split("\n")
    for line in lines:
        if not line.strip():
            continue
        sname, field, val = line.split()
        cls = getattr(B, sname)
        if field == "size":
            assert ctypes.sizeof(cls) == int(val), line
        else:
            assert getattr(cls, field).offset == int(val), line


def _grid(B, N=4096, dtype=None, length=6.283185307179586):
    g = B.at_grid()
    g.dim, g.bc = 1, B.AT_BC_PERIODIC
    g.dtype = B.AT_F64 if dtype is None else dtype
    g.n[0], g.n[1], g.n[2] = N, 1, 1
    g.length[0] = length
    return g


def test_workspace_bytes_and_validation(B):
    g = _grid(B)
    nb = B.at_workspace_bytes(g, 16, 2, 2)
    # state + ring + flags + control at least
    assert nb >= 4096 * 8 + 8 * 16 * 2 * 16 + 16 * 2 * 8
    assert nb % 256 == 0
    assert B.at_workspace_bytes(g, 3, 2, 2) == 0 and "N % P" in B.at_last_error()
    assert B.at_workspace_bytes(g, 16, 3, 2) == 0 and "order" in B.at_last_error()
    assert B.at_workspace_bytes(g, 16, 2, 17) == 0 and "L must" in B.at_last_error()
    assert B.at_workspace_bytes(_grid(B, N=4096 + 16 * 2), 16, 2, 2) == 0   # M = 258
    assert B.at_workspace_bytes(_grid(B, dtype=7), 16, 2, 2) == 0
    g.dim = 3
    assert B.at_workspace_bytes(g, 16, 2, 2) == 0


def test_3d_workspace_and_subdomain_count_limit(B):
    """A 3D grid's workspace is sized on the host; more than 2^31 - 1
    subdomains are refused (the kernel keeps subdomain indices in 32 bits)."""
    g = _grid(B, dtype=B.AT_F32)
    g.dim = 3
    for a, (n, m) in enumerate([(64, 32), (64, 32), (32, 8)]):
        g.n[a], g.sub[a], g.length[a] = n, m, 6.283185307179586
    assert B.at_workspace_bytes(g, 2 * 2 * 4, 2, 2) > 0
    for a, (n, m) in enumerate([(4 << 11, 4), (2 << 11, 2), (3 << 9, 3)]):
        g.n[a], g.sub[a] = n, m
    assert B.at_workspace_bytes(g, 1 << 31, 2, 2) == 0 and "2^31" in B.at_last_error()


def test_3d_steps_per_pass_validation(B):
    """3D passes of several levels: at most L + 1 (and 4) levels, and rows of
    a power-of-two sub[0] (4 .. 128) so a row's column groups lie in one warp."""
    g = _grid(B, dtype=B.AT_F32)
    g.dim = 3
    for a, (n, m) in enumerate([(64, 32), (64, 32), (32, 8)]):
        g.n[a], g.sub[a], g.length[a] = n, m, 6.283185307179586
    for spp in (0, 1, 2, 3):
        g.steps_per_pass = spp
        assert B.at_workspace_bytes(g, 2 * 2 * 4, 2, 2) > 0
    g.steps_per_pass = 4                                   # > L + 1
    assert B.at_workspace_bytes(g, 2 * 2 * 4, 2, 2) == 0 and "steps_per_pass" in B.at_last_error()
    assert B.at_workspace_bytes(g, 2 * 2 * 4, 2, 3) > 0
    g.steps_per_pass = 5                                   # > 4 levels of registers
    assert B.at_workspace_bytes(g, 2 * 2 * 4, 2, 6) == 0 and "steps_per_pass" in B.at_last_error()
    g.steps_per_pass = 2
    for a, (n, m) in enumerate([(48, 12), (64, 32), (32, 8)]):   # sub[0] = 12: not a power of two
        g.n[a], g.sub[a] = n, m
    assert B.at_workspace_bytes(g, 4 * 2 * 4, 2, 2) == 0 and "power of two" in B.at_last_error()
    g.steps_per_pass = 1
    assert B.at_workspace_bytes(g, 4 * 2 * 4, 2, 2) > 0


def test_create_rejects_bad_arguments_on_the_host(B):
    g = _grid(B)
    dx = 6.283185307179586 / 4096
    rc, h = B.at_create(g, 16, 2, 2, 0.02, 1e-6)       # no workspace
    assert rc == B.AT_ERR_ARG and not h.value
    rc, _ = B.at_create(g, 16, 2, 2, 0.02, -1.0)
    assert rc == B.AT_ERR_ARG
    rc, _ = B.at_create(g, 16, 2, 2, -0.1, 1e-6)
    assert rc == B.AT_ERR_ARG
    rc, _ = B.at_create(g, 16, 2, 2, 0.02, 0.6 * dx * dx / 0.02)   # nu dt/dx^2 = 0.6 > 1/2
    assert rc == B.AT_ERR_UNSTABLE
    rc, _ = B.at_create(g, 16, 4, 2, 0.02, 0.4 * dx * dx / 0.02)   # 0.4 > 3/8 for order 4
    assert rc == B.AT_ERR_UNSTABLE


def test_product_path_has_no_cpu_fallback():
    """The package refuses to run without the CUDA library and never imports
    the oracle."""
    import paper_1911_05769_gb300 as pkg
    src_dir = os.path.dirname(pkg.__file__)
    for name in os.listdir(src_dir):
        if name.endswith(".py"):
            text = open(os.path.join(src_dir, name)).read()
            assert "import oracle" not in text and "from oracle" not in text, name


def _instances(B, specs):
    arr = (B.at_instance * len(specs))()
    for a, (n, L, nu, dt) in zip(arr, specs):
        a.n, a.L, a.bc = n, L, B.AT_BC_EXACT_TANH
        a.length, a.origin, a.nu, a.dt = 6.283185307179586, -3.141592653589793, nu, dt
        a.tanh_a, a.tanh_c = 0.1, 0.2
    return arr


def test_batch_workspace_bytes_and_validation(B):
    g = B.at_grid()
    g.dim, g.dtype = 1, B.AT_F32
    ok = _instances(B, [(1024, 1, 0.01, 1e-5), (512, 3, 0.02, 1e-5)])
    nb = B.at_batch_workspace_bytes(g, ok, 256, 2)
    P = (1024 + 512) // 256
    # state + ring (T = 16 for L = 3, s = 2) + flags + subdomain and instance records
    assert nb >= 1536 * 4 + 16 * P * 2 * 16 + P * 2 * 8 + P * 64 + 2 * 64
    assert nb % 256 == 0
    assert B.at_batch_workspace_bytes(g, _instances(B, [(1000, 1, 0.01, 1e-5)]), 256, 2) == 0
    assert "multiple of M" in B.at_last_error()
    assert B.at_batch_workspace_bytes(g, _instances(B, [(1024, 17, 0.01, 1e-5)]), 256, 2) == 0
    assert B.at_batch_workspace_bytes(g, _instances(B, [(1024, 1, 0.0, 1e-5)]), 256, 2) == 0
    assert "nu > 0" in B.at_last_error()
    assert B.at_batch_workspace_bytes(g, ok, 258, 2) == 0
    assert B.at_batch_workspace_bytes(g, ok, 256, 3) == 0
    # nu dt / dx^2 = 0.01 * 1e-2 / (2 pi / 1024)^2 > 1/2
    assert B.at_batch_workspace_bytes(g, _instances(B, [(1024, 1, 0.01, 1e-2)]), 256, 2) == 0
    assert "exceeds" in B.at_last_error()
    g.steps_per_pass = 5                                  # above max L + 1 = 4
    assert B.at_batch_workspace_bytes(g, ok, 256, 2) == 0
    g.steps_per_pass = 0
    g.forcing_amp = 0.1
    assert B.at_batch_workspace_bytes(g, ok, 256, 2) == 0 and "unforced" in B.at_last_error()
    g.forcing_amp = 0.0
    rc, h = B.at_create_batch(g, ok, 256, 2)              # no workspace
    assert rc == B.AT_ERR_ARG and not h.value
