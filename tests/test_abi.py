"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/pop.h declares, and its host-only logic (CSR validation, error paths
before any GPU work) behaves as documented.  No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pop.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1904_02863_gb300 import binding, build
    build.build()
    return binding.load_library()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pop_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("pop_create", "pop_destroy", "pop_load_events", "pop_load_injections", "pop_loglik",
                 "pop_autotune", "pop_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1904_02863_gb300 import binding
    syms = declared_symbols()
    for name in syms:
        assert hasattr(lib, name), f"libpop.so does not export {name}"
    assert set(syms) == set(binding.EXPORTS), "binding.EXPORTS out of sync with include/pop.h"


def test_version_and_status_strings(lib):
    from paper_1904_02863_gb300 import binding as B
    assert B.pop_version() >= 10000
    assert B.status_string(B.POP_EINVAL) == "POP_EINVAL"
    assert B.status_string(B.POP_ETIMEOUT) == "POP_ETIMEOUT"
    assert B.status_string(12345) == "POP_UNKNOWN"


@pytest.mark.parametrize("offsets,n_dims,ok,needle", [
    ([0, 3, 7], 6, True, ""),
    ([0, 3, 7], 7, True, ""),
    ([1, 3, 7], 6, False, "offsets[0]"),
    ([0, 3, 3], 6, False, ">= 1 sample"),
    ([0, 5, 4], 6, False, ">= 1 sample"),
    ([0, 3, 7], 5, False, "n_dims"),
])
def test_validate_events_host_logic(lib, offsets, n_dims, ok, needle):
    from paper_1904_02863_gb300 import binding as B
    rc, msg = B.pop_validate_events(len(offsets) - 1, np.array(offsets), n_dims)
    assert (rc == B.POP_OK) == ok
    assert needle in msg


def test_validate_rejects_empty_catalog(lib):
    from paper_1904_02863_gb300 import binding as B
    rc, msg = B.pop_validate_events(0, np.array([0]), 6)
    assert rc == B.POP_EINVAL and "n_events" in msg


def test_null_context_is_rejected(lib):
    from paper_1904_02863_gb300 import binding as B
    assert lib.pop_loglik(None, 1, 11, None, 0, None, None, None, None, 0) == B.POP_EINVAL
    assert lib.pop_destroy(None) == B.POP_OK


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1904_02863_gb300 import binding as B
    with pytest.raises(B.PopError) as e:
        B.pop_create(0)
    assert e.value.status == B.POP_ECUDA


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1904_02863_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "pop_oracle" not in src, f


def test_noalloc_wrapper_takes_cuda_tensors_of_one_device_only():
    """The no-allocation wrapper refuses numpy arrays and CPU tensors before it reaches the library
    (the device and stream it runs on are taken from the tensors)."""
    import torch
    from paper_1904_02863_gb300 import binding
    off = torch.tensor([0, 2], dtype=torch.int64)
    th, pr = torch.zeros(2, 6, dtype=torch.float64), torch.ones(2, dtype=torch.float64)
    lam = torch.zeros(1, 11, dtype=torch.float64)
    out = (torch.empty(1, dtype=torch.float64),) * 3 + (torch.empty(1, dtype=torch.int32),)
    with pytest.raises(ValueError):
        binding.pop_loglik_f64_noalloc(off, th, pr, 10, th, pr, lam, out)
    with pytest.raises(ValueError):
        binding.pop_loglik_f64_noalloc(off.numpy(), th, pr, 10, th, pr, lam, out)
