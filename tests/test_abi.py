"""The C-ABI library loads and exports every symbol include/dc_fmm.h
declares; the ctypes mirrors of its structs have the C layout.  CPU only:
no compute call is made."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dc_fmm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dc_build_tree", "dc_solve_density", "dc_render_viewport", "dc_create",
                 "dc_destroy", "dc_eval_points"):
        assert must in names


def test_library_exports_every_declared_symbol(dcmod):
    lib = dcmod.lib
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", dcmod.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (dc_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_struct_layouts_match_header(dcmod):
    """Compile a tiny C program against the header and compare sizeof and
    offsets with the ctypes mirrors."""
    P = dcmod
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "dc_fmm.h"
int main(void){
 printf("%zu %zu %zu %zu %zu\n", sizeof(dc_options), sizeof(dc_sizes), sizeof(dc_solve_stats),
        sizeof(dc_viewport), sizeof(dc_render_stats));
 printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", offsetof(dc_options, stream), offsetof(dc_options, domain),
        offsetof(dc_solve_stats, p2p_pairs), offsetof(dc_render_stats, eval_flops),
        offsetof(dc_solve_stats, warm_resid), offsetof(dc_solve_stats, ms_warm),
        offsetof(dc_options, p_inner), offsetof(dc_options, inner_tol), offsetof(dc_options, m2l_engine));
 printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dc_subdivide_options), sizeof(dc_subdivide_stats),
        offsetof(dc_subdivide_options, label_ratio), offsetof(dc_subdivide_stats, ms_solve),
        offsetof(dc_options, coarse_max), offsetof(dc_solve_stats, true_rel_resid),
        offsetof(dc_options, adapt_max_len), offsetof(dc_options, eval_tile));
 printf("%zu %zu %zu\n", offsetof(dc_options, aa_levels), offsetof(dc_render_stats, aa_pixels),
        offsetof(dc_render_stats, ms_aa));
 printf("%zu %zu %zu %zu\n", sizeof(dc_view_options), sizeof(dc_view_stats), offsetof(dc_view_options, label_ratio),
        offsetof(dc_view_stats, ms_total));
 return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    sizes = list(map(int, lines[0].split()))
    offs = list(map(int, lines[1].split()))
    import ctypes
    assert sizes == [ctypes.sizeof(P.dc_options), ctypes.sizeof(P.dc_sizes),
                     ctypes.sizeof(P.dc_solve_stats), ctypes.sizeof(P.dc_viewport),
                     ctypes.sizeof(P.dc_render_stats)]
    assert offs == [P.dc_options.stream.offset, P.dc_options.domain.offset,
                    P.dc_solve_stats.p2p_pairs.offset, P.dc_render_stats.eval_flops.offset,
                    P.dc_solve_stats.warm_resid.offset, P.dc_solve_stats.ms_warm.offset,
                    P.dc_options.p_inner.offset, P.dc_options.inner_tol.offset,
                    P.dc_options.m2l_engine.offset]
    sub = list(map(int, lines[2].split()))
    assert sub == [ctypes.sizeof(P.dc_subdivide_options), ctypes.sizeof(P.dc_subdivide_stats),
                   P.dc_subdivide_options.label_ratio.offset, P.dc_subdivide_stats.ms_solve.offset,
                   P.dc_options.coarse_max.offset, P.dc_solve_stats.true_rel_resid.offset,
                   P.dc_options.adapt_max_len.offset, P.dc_options.eval_tile.offset]
    aa = list(map(int, lines[3].split()))
    assert aa == [P.dc_options.aa_levels.offset, P.dc_render_stats.aa_pixels.offset,
                  P.dc_render_stats.ms_aa.offset]
    vw = list(map(int, lines[4].split()))
    assert vw == [ctypes.sizeof(P.dc_view_options), ctypes.sizeof(P.dc_view_stats),
                  P.dc_view_options.label_ratio.offset, P.dc_view_stats.ms_total.offset]


def test_defaults_and_status_strings(dcmod):
    o = dcmod.default_options()
    assert (o.form, o.g, o.s_per_panel, o.p) == (dcmod.DC_FORM_FMM32, 16, 80, 24)
    assert dcmod.lib.dc_abi_version() == 1
    assert dcmod.lib.dc_status_string(dcmod.DC_ERR_STATE) == b"call out of order"


def test_create_rejects_bad_options_without_touching_the_gpu(dcmod):
    import ctypes
    o = dcmod.default_options(g=0)
    h = ctypes.c_void_p()
    st = dcmod.lib.dc_create(ctypes.byref(h), ctypes.byref(o))
    assert st == dcmod.DC_ERR_ARG
    assert b"g must be" in dcmod.lib.dc_last_error(None)
    assert not h.value


def test_null_context_is_rejected(dcmod):
    assert dcmod.lib.dc_solve_density(None, None, None) == dcmod.DC_ERR_ARG
    dcmod.lib.dc_destroy(None)
