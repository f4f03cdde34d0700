"""The C ABI used from C: a C99 program compiled with gcc against include/bfgc.h and linked
against libbfgc.so calls the host-only entry points (plan, options, plan info, workspace
sizes, argument errors, status strings) and checks what the header documents.  No kernel is
launched and no device is needed."""
import os
import shutil
import subprocess

import pytest

from paper_1605_02178_gb300 import bfgc as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "bfgc.h"

#define CHECK(c) do { if (!(c)) { printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main(void) {
    bf_gc_plan_t p = NULL;
    bf_gc_info info;
    size_t fwd = 0, bwd = 0, cs;
    CHECK(bf_gc_plan(2160, 3840, 10.0, 50.0, 20, &p) == BF_OK && p != NULL);
    CHECK(bf_gc_plan_info(p, &info) == BF_OK);
    CHECK(info.H == 2160 && info.W == 3840 && info.N == 20 && info.C == 22 && info.R == 30);
    CHECK(info.form == BF_FORM_PLAIN && info.precision == BF_PREC_FP32);
    CHECK(info.fit_err > 0.0 && info.fit_err < 1e-6);         /* sigma_r = 50, N = 20: converged */
    cs = ((size_t)2160 * 3840 + 63) / 64 * 64;
    CHECK(bf_gc_workspace_size(p, &fwd, &bwd) == BF_OK);
    /* plain: two sets of FP32 planes, then the FP64 refinement list (one index per pixel) */
    CHECK(fwd == 256 + 2 * 22 * cs * sizeof(float) + (size_t)2160 * 3840 * 4);
    CHECK(bf_gc_plan_set(p, BF_OPT_FORM, BF_FORM_FUSED) == BF_OK);
    CHECK(bf_gc_workspace_size(p, &fwd, NULL) == BF_OK);
    CHECK(fwd == 256 + 22 * cs * sizeof(float) + (size_t)2160 * 3840 * 4);   /* fused FP32: one set */
    CHECK(bf_gc_plan_set(p, BF_OPT_FORM, BF_FORM_AUTO) == BF_OK);
    CHECK(bf_gc_plan_info(p, &info) == BF_OK && info.form == BF_FORM_FUSED);   /* R = 30 <= 140 */
    CHECK(bf_gc_plan_set(p, BF_OPT_PRECISION, BF_PREC_BF16) == BF_OK);
    CHECK(bf_gc_plan_info(p, &info) == BF_OK && info.form == BF_FORM_FUSED_TC);
    CHECK(bf_gc_plan_set(p, 99, 1.0) == BF_ERR_INVALID_ARG);
    CHECK(bf_gc_plan_set(p, BF_OPT_FORM, 5.0) == BF_ERR_INVALID_ARG);
    CHECK(bf_gc_forward(p, NULL, NULL, NULL, 0, NULL) == BF_ERR_INVALID_ARG);
    CHECK(strlen(bf_status_string(BF_ERR_WORKSPACE)) > 0);
    bf_gc_plan_destroy(p);
    CHECK(bf_gc_plan(0, 10, 1.0, 10.0, 4, &p) == BF_ERR_INVALID_ARG && p == NULL);
    printf("ok\n");
    return 0;
}
"""


def test_c_program_uses_the_abi(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = B.lib()                                   # builds libbfgc.so if needed
    assert lib is not None
    libdir = os.path.dirname(B.LIB_PATH)
    src = tmp_path / "abi.c"
    exe = tmp_path / "abi"
    src.write_text(PROGRAM)
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", cuda_inc, str(src), "-o", str(exe), "-L", libdir, "-lbfgc", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
