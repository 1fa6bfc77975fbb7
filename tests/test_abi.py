"""The C ABI: every entry point declared in include/gpbo.h is exported by the built
library, the binding loads it, and without a usable sm_103 GPU the library refuses
to run (no CPU fallback).  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpbo.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|int64_t|char|void)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2403_08131_b300 import build
    return build.build()


def test_header_declares_the_four_calls():
    names = declared_functions()
    for want in ["gp_fit", "gp_posterior_ei", "interdep_screen", "search_step", "gpbo_create", "gpbo_destroy"]:
        assert want in names


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(declared_functions()) <= exported


def test_built_for_sm103a(libpath):
    log = open(os.path.join(os.path.dirname(libpath), "build.log")).read()
    assert "arch=compute_103a,code=sm_103a" in log
    assert "tcgen05" in open(os.path.join(ROOT, "paper_2403_08131_b300", "csrc", "score_tc.cu")).read()


def test_binding_loads_and_reports_status_strings(libpath):
    from paper_2403_08131_b300 import gpbo
    assert gpbo.strerror(0) == "ok"
    assert "positive definite" in gpbo.strerror(gpbo.GPBO_ENOTSPD)


def test_no_gpu_means_refusal_not_fallback(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2403_08131_b300 import gpbo
    with pytest.raises(gpbo.GpboError) as e:
        gpbo.Context(0)
    assert e.value.code == gpbo.GPBO_ENOTSUP
