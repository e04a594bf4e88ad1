"""Host-side checks of the C-ABI library that need no GPU: it loads, exports every function the
header declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cbessfm.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cbessfm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_14489_gb300 import cbessfm
    return cbessfm


def test_library_exports_every_declared_function(lib):
    names = _declared_functions()
    assert "cbessfm_backpropagate" in names and "cbessfm_plan_create" in names
    so = ctypes.CDLL(lib._LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_version_string(lib):
    assert "sm_103a" in lib.version()


@pytest.mark.parametrize("kw,msg", [
    (dict(bands=0), "bands"), (dict(bands=17), "bands"), (dict(steps=-1), "steps"),
    (dict(ratio=1.5), "ratio"), (dict(ratio=-0.1), "ratio"), (dict(n_fft=100), "n_fft"),
    (dict(n_fft=8), "n_fft"), (dict(n_fft=4096), "n_fft"), (dict(ntaps=4), "ntaps"),
    (dict(ntaps=129), "ntaps"), (dict(overlap=3), "overlap"), (dict(overlap=256), "overlap"),
])
def test_plan_create_rejects_invalid_arguments(lib, kw, msg):
    import numpy as np
    args = dict(bands=1, steps=1, ratio=0.5, ntaps=5, n_fft=256, overlap=64)
    args.update(kw)
    taps = np.zeros((max(args["steps"], 0), max(args["bands"], 0), max(args["bands"], 0),
                     args["ntaps"]), np.float32)
    link = lib.make_link(-21.7e-27, 80e3, 1, 64e9)
    h = ctypes.c_void_p()
    st = lib.lib().cbessfm_plan_create(
        ctypes.byref(link), args["bands"], args["steps"], args["ratio"],
        taps.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if taps.size else None,
        args["ntaps"], args["n_fft"], args["overlap"], 0, ctypes.byref(h))
    assert st == lib.ERR_INVALID_ARG
    assert msg in lib.lib().cbessfm_last_error().decode()
    assert not h.value


def test_invalid_link_and_null_arguments(lib):
    link = lib.make_link(-21.7e-27, 80e3, 1, 0.0)
    h = ctypes.c_void_p()
    assert lib.lib().cbessfm_plan_create(ctypes.byref(link), 1, 0, 0.5, None, 1, 64, 16, 0,
                                         ctypes.byref(h)) == lib.ERR_INVALID_ARG
    assert lib.lib().cbessfm_plan_create(None, 1, 0, 0.5, None, 1, 64, 16, 0,
                                         ctypes.byref(h)) == lib.ERR_INVALID_ARG
    assert lib.lib().cbessfm_backpropagate(None, None, None, 10, 1, None) == lib.ERR_INVALID_ARG
    assert lib.lib().cbessfm_backpropagate_host(None, None, None, None, None, 10, 1, 0,
                                                None) == lib.ERR_INVALID_ARG
    assert lib.lib().cbessfm_backpropagate_streamed(None, None, None, None, 0, 10, 1,
                                                    None) == lib.ERR_INVALID_ARG
    assert lib.lib().cbessfm_set_nlpr_mode(None, 1) == lib.ERR_INVALID_ARG
    assert lib.lib().cbessfm_plan_destroy(None) == lib.OK


@pytest.mark.parametrize("kw,msg", [
    (dict(bands=0), "bands"), (dict(steps=0), "steps"), (dict(ntaps=4), "ntaps"),
    (dict(grid=3), "grid"), (dict(spans_per_step=0), "spans_per_step"),
    (dict(spans_per_step=3), "spans_per_step"), (dict(alpha=-1.0), "alpha"),
])
def test_analytic_taps_rejects_invalid_arguments(lib, kw, msg):
    import numpy as np
    args = dict(bands=3, steps=2, ntaps=5, grid=16, spans_per_step=1, alpha=4.6e-5)
    args.update(kw)
    link = lib.make_link(-21.7e-27, 80e3, 4, 64e9, gamma=1.3e-3, alpha=args["alpha"])
    taps = np.zeros(4096)
    pw = np.ones(8)
    st = lib.lib().cbessfm_analytic_taps(ctypes.byref(link), args["bands"], args["steps"],
                                         args["spans_per_step"], pw.ctypes.data, args["ntaps"],
                                         args["grid"], taps.ctypes.data, None)
    assert st == lib.ERR_INVALID_ARG
    assert msg in lib.lib().cbessfm_last_error().decode()


def test_every_entry_point_rejects_a_null_handle_without_a_device(lib):
    """Each call that takes a plan or batch validates it before any CUDA call: a NULL handle
    (or NULL output pointer) is INVALID_ARG with a message, never a crash; destroy(NULL) is OK."""
    L, E, P = lib.lib(), lib, None
    size = ctypes.c_size_t()
    n_groups, n_items = ctypes.c_int(), ctypes.c_longlong()
    checks = {
        "set_coeffs": lambda: L.cbessfm_set_coeffs(P, P, 0, P),
        "set_ratio": lambda: L.cbessfm_set_ratio(P, ctypes.c_double(0.5), P),
        "grad_workspace_size": lambda: L.cbessfm_grad_workspace_size(P, 100, 1, ctypes.byref(size)),
        "backpropagate_checkpointed": lambda: L.cbessfm_backpropagate_checkpointed(
            P, P, P, 100, 1, P, 0, P),
        "grad": lambda: L.cbessfm_grad(P, P, P, P, P, P, 0, 100, 1, P),
        "batch_create": lambda: L.cbessfm_batch_create(P, 1, P),
        "batch_run": lambda: L.cbessfm_batch_run(P, P),
        "batch_info": lambda: L.cbessfm_batch_info(P, ctypes.byref(n_groups), ctypes.byref(n_items)),
        "batch_run_noalloc": lambda: L.cbessfm_batch_run_noalloc(P, 1, P),
        "streamed_workspace_size": lambda: L.cbessfm_streamed_workspace_size(
            P, 100, 1, ctypes.byref(size)),
        "get_status": lambda: L.cbessfm_get_status(P, P),
        "set_wait_limit": lambda: L.cbessfm_set_wait_limit(P, 0),
        "measure_fp32_peak": lambda: L.cbessfm_measure_fp32_peak(1, P, P, P),
    }
    for name, call in checks.items():
        st = call()
        assert st == E.ERR_INVALID_ARG, (name, st)
        assert L.cbessfm_last_error(), name
    assert L.cbessfm_batch_destroy(P) == E.OK


def test_plan_create_rejects_more_invalid_arguments(lib):
    """Step count cap, a NaN ratio, an unknown storage type, missing taps and broken links."""
    import numpy as np
    L = lib.lib()
    taps = np.zeros((1, 1, 1, 5), np.float32)
    tp = taps.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    good = lib.make_link(-21.7e-27, 80e3, 1, 64e9)
    h = ctypes.c_void_p()

    def create(link, steps=1, ratio=0.5, coeffs=tp, storage=0):
        return L.cbessfm_plan_create(ctypes.byref(link), 1, steps, ratio, coeffs, 5, 256, 64,
                                     storage, ctypes.byref(h))

    for kw, msg in [(dict(steps=4097), "steps"), (dict(ratio=float("nan")), "ratio"),
                    (dict(storage=7), "storage"), (dict(coeffs=None), "coeffs")]:
        assert create(good, **kw) == lib.ERR_INVALID_ARG, kw
        assert msg in L.cbessfm_last_error().decode(), kw
        assert not h.value
    for link, msg in [(lib.make_link(-21.7e-27, 0.0, 1, 64e9), "span_length"),
                      (lib.make_link(-21.7e-27, 80e3, 0, 64e9), "span_length"),
                      (lib.make_link(float("inf"), 80e3, 1, 64e9), "beta2"),
                      (lib.make_link(-21.7e-27, 80e3, 1, float("nan")), "sample_rate")]:
        assert create(link) == lib.ERR_INVALID_ARG, msg
        assert msg in L.cbessfm_last_error().decode(), msg


def test_plan_and_batch_close_idempotently_as_context_managers(lib):
    """Plan and Batch release their handle on leaving a `with` block; close() on a released (NULL)
    handle is a no-op, so an explicit close inside the block and __del__ afterwards are safe."""
    for cls in (lib.Plan, lib.Batch):
        obj = object.__new__(cls)
        obj._h = ctypes.c_void_p()
        with obj as same:
            assert same is obj
            obj.close()
        assert not obj._h.value
        obj.close()
        obj.__del__()


_GUARD_CHILD = r"""
import ctypes, resource, sys
so = ctypes.CDLL(sys.argv[1])
so.cbessfm_last_error.restype = ctypes.c_char_p
job = ctypes.create_string_buffer(64)                 # one zeroed job; never read (see below)
out = ctypes.c_void_p()
vm = int([l.split()[1] for l in open("/proc/self/status") if l.startswith("VmSize")][0]) * 1024
resource.setrlimit(resource.RLIMIT_AS, (vm + (256 << 20), resource.RLIM_INFINITY))
st = so.cbessfm_batch_create(job, (1 << 31) - 1, ctypes.byref(out))
print(st, so.cbessfm_last_error().decode(), out.value)
"""


def test_host_allocation_failure_is_a_status_not_an_exception(lib):
    """No C++ exception crosses the ABI: under an address-space limit, batch_create's first host
    container (one descriptor per job, here 2^31 - 1 of them, allocated before any job is read)
    cannot be allocated, and the call returns CBESSFM_ERR_OOM with a message and no batch instead
    of terminating the process.  Run in a child process, which the limit confines."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _GUARD_CHILD, lib._LIB_PATH],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    st, rest = r.stdout.strip().split(" ", 1)
    assert int(st) == lib.ERR_OOM, r.stdout
    assert "host resources exhausted" in rest and rest.endswith("None"), r.stdout


def test_batch_jobs_are_validated_before_the_library_call(lib):
    """A job's x and y must be (L, 2) complex64 (or (L, 4) 16-bit) CUDA tensors of equal shape:
    host tensors, or a (batch, L, 2) field that a job would cut to its first realization, are
    refused with ValueError before cbessfm_batch_create runs."""
    import torch
    plan = object.__new__(lib.Plan)
    plan._h = ctypes.c_void_p()
    plan.storage = lib.STORAGE_C64
    x = torch.zeros((64, 2), dtype=torch.complex64)
    for bad in [(x, x), (x.reshape(1, 64, 2), x.reshape(1, 64, 2))]:
        with pytest.raises(ValueError, match="job 0: x must be a contiguous"):
            lib.Batch([(plan, *bad)])


def test_field_checks_of_the_binding(lib):
    """The binding refuses fields whose size the library would misread: wrong dtype for the
    plan's storage, a last dimension other than 2 (complex64) or 4 (16-bit), another rank, a
    non-contiguous view, an output of another shape, or host/device memory in the wrong place."""
    import torch
    plan = object.__new__(lib.Plan)
    plan._h = ctypes.c_void_p()
    plan.storage = lib.STORAGE_C64
    x = torch.zeros((3, 40, 2), dtype=torch.complex64)
    assert plan._field(x, "x", host=True) == (3, 40)
    assert plan._field(x[0], "x", host=True) == (1, 40)
    assert plan._field(x, "out", like=x, host=True) == (3, 40)
    bad = [x.to(torch.complex128), x.reshape(3, 80, 1), x.reshape(240), x[:, ::2],
           torch.zeros((3, 40, 4), dtype=torch.float16)]
    for t in bad:
        with pytest.raises(ValueError, match="x must be a contiguous"):
            plan._field(t, "x", host=True)
    with pytest.raises(ValueError, match="the same as x"):
        plan._field(x[:2], "out", like=x, host=True)
    with pytest.raises(ValueError, match="CUDA tensor"):
        plan._field(x, "x")
    plan.storage = lib.STORAGE_F16X4
    assert plan._field(torch.zeros((40, 4), dtype=torch.float16), "x", host=True) == (1, 40)
    with pytest.raises(ValueError, match="float16"):
        plan._field(x, "x", host=True)
    # the public calls check before any library call
    with pytest.raises(ValueError, match="h_in must be a contiguous torch.float16 host tensor"):
        plan.backpropagate_host(x, x, x, x)
    plan.storage = lib.STORAGE_C64
    with pytest.raises(ValueError, match="d_in must be a contiguous torch.complex64 CUDA"):
        plan.backpropagate_host(x, x, x, x)
    with pytest.raises(ValueError, match="x must be a contiguous torch.complex64 CUDA"):
        plan.backpropagate(x)


def test_block_count_helpers_do_not_overflow(tmp_path):
    """Every entry point refuses more than 2^31 - 1 blocks before it forms a size from
    n_samples * batch; the helpers it uses are exact at the int64 and int32 limits."""
    import subprocess
    src = os.path.join(ROOT, "tests", "block_count_check.cc")
    inc = os.path.join(ROOT, "paper_2409_14489_gb300", "csrc")
    exe = str(tmp_path / "block_count_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Werror", "-I", inc, src, "-o", exe],
                   check=True, capture_output=True, text=True, timeout=120)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout


def test_set_coeffs_checks_the_tap_shape(lib):
    """set_coeffs refuses taps of another shape than the plan's [steps][bands][bands][ntaps]
    before the library reads them (it would read past a shorter array)."""
    import numpy as np
    plan = object.__new__(lib.Plan)
    plan._h = ctypes.c_void_p()
    plan.steps, plan.bands, plan.ntaps = 2, 3, 5
    for shape in [(2, 3, 3, 3), (1, 3, 3, 5), (90,)]:
        with pytest.raises(ValueError, match=r"coeffs must have shape \(2, 3, 3, 5\)"):
            plan.set_coeffs(np.zeros(shape, np.float32))


def test_workspace_must_be_device_memory(lib):
    """A workspace is written by the kernels: a host tensor (whose address would fault the
    device) or a strided view is refused before the library call."""
    import torch
    for ws in [torch.zeros(256, dtype=torch.uint8), torch.zeros(512, dtype=torch.uint8)[::2]]:
        with pytest.raises(ValueError, match="workspace must be a contiguous CUDA tensor"):
            lib.Plan._workspace(ws)
