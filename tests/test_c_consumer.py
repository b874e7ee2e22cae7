"""The boundary is a plain C ABI: a C99 program that includes include/ozg.h and include/ozg_blas.h
compiles with gcc -std=c99 -pedantic -Wall -Wextra -Werror (no C++ or CUDA types leak into the
headers), links against the built libozg.so, and gets the documented answers from calls that
need no GPU: strerror texts, xerbla-numbered argument errors, OZG_ERR_INVALID for a null
context, and the shim's mode parsing.  With no GPU visible ozg_create reports a runtime error
and leaves no context behind."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ozg.h"
#include "ozg_blas.h"

static int fails = 0;
static void expect(int got, int want, const char* what) {
  if (got != want) {
    printf("FAIL %s: got %d, want %d\n", what, got, want);
    ++fails;
  }
}

int main(int argc, char** argv) {
  const double one[2] = {1.0, 0.0};
  ozg_ctx* ctx = NULL;
  int rc;
  (void)argc;
  expect(strlen(ozg_strerror(0)) > 0, 1, "strerror(0)");
  expect(ozg_dgemm(NULL, 'N', 'N', -1, 4, 4, 1.0, NULL, 4, NULL, 4, 0.0, NULL, 4, 7, NULL), -3, "m < 0");
  expect(ozg_dgemm(NULL, 'N', 'N', 4, 4, 4, 1.0, NULL, 3, NULL, 4, 0.0, NULL, 4, 7, NULL), -8, "lda");
  expect(ozg_dgemm(NULL, 'N', 'N', 4, 4, 4, 1.0, NULL, 4, NULL, 4, 0.0, NULL, 4, 19, NULL), -14, "slices");
  expect(ozg_dgemm(NULL, 'N', 'N', 4, 4, 4, 1.0, NULL, 4, NULL, 4, 0.0, NULL, 4, 7, NULL), OZG_ERR_INVALID,
         "null context");
  expect(ozg_zgemm(NULL, 'C', 'N', 4, 4, 6, one, NULL, 5, NULL, 6, one, NULL, 4, 7, NULL), -8, "zgemm lda");
  expect(ozg_blas_parse_mode("dgemm"), OZG_NATIVE, "mode dgemm");
  expect(ozg_blas_parse_mode("fp64_int8_9"), 9, "mode fp64_int8_9");
  expect(ozg_blas_parse_mode("fp64_int8_19"), 0, "mode fp64_int8_19");
  if (strcmp(argv[1], "nogpu") == 0) {
    rc = ozg_create(&ctx, 0);
    expect(rc > 0, 1, "ozg_create without a GPU");
    expect(ctx == NULL, 1, "no context without a GPU");
  }
  printf("%s\n", fails ? "FAILED" : "OK");
  return fails != 0;
}
"""


def test_c99_program_builds_links_and_gets_documented_answers(tmp_path):
    from paper_2503_22875_gb300 import build
    build.build()
    libdir = os.path.dirname(build.LIB)
    blas = os.path.join(libdir, "libozg_blas.so")
    assert os.path.exists(build.LIB) and os.path.exists(blas)
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = str(tmp_path / "consumer")
    subprocess.check_call(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", exe, "-L", libdir, "-lozg", "-lozg_blas",
                           f"-Wl,-rpath,{libdir}"])
    try:
        import torch
        gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        gpu = False
    r = subprocess.run([exe, "gpu" if gpu else "nogpu"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr
