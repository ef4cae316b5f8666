"""The C-ABI library builds for sm_103a, loads, and exports every symbol its header declares.

CPU only: no compute call is made (there may be no GPU).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "helm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"#define HELM_API.*", "", text)
    return sorted(set(re.findall(r"HELM_API\s+[\w\s\*]*?\b(\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2308_11469_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    names = _declared()
    for want in ["helm_plan_create", "helm_plan_destroy", "helm_plan_info", "helm_solve",
                 "poisson_vcycle", "helm_status_str", "helm_batch_create", "helm_batch_submit",
                 "helm_batch_step", "helm_batch_poll"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(lib):
    from paper_2308_11469_gb300 import binding
    binding.load()
    assert set(_declared()) == set(binding._SIGS)
    for name in _declared():
        assert callable(getattr(binding, name))


def test_status_strings_without_gpu(lib):
    from paper_2308_11469_gb300 import binding
    assert binding.helm_status_str(0) == "HELM_CONVERGED"
    assert binding.helm_status_str(2) == "HELM_DIVERGED"
    assert binding.helm_status_str(-1) == "HELM_EINVAL"
    assert binding.helm_status_str(99) == "HELM_UNKNOWN"


def test_null_arguments_are_rejected_without_touching_the_device(lib):
    lib.helm_plan_create.restype = ctypes.c_int
    assert lib.helm_plan_create(None, 2, None, ctypes.c_double(0.1), ctypes.c_double(1.0), 0, 1, None) == -1
    lib.helm_plan_info.restype = ctypes.c_int
    assert lib.helm_plan_info(None, None, None, None, None) == -1
    lib.helm_batch_poll.restype = ctypes.c_int
    assert lib.helm_batch_poll(None, ctypes.c_uint64(1), None, None, None, None) == -1


def test_library_is_built_for_sm_103a(lib):
    from paper_2308_11469_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
