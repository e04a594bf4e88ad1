"""The C-ABI from a plain C99 program (tests/c_abi_example.c, no Python in the data path): the
header compiles as C99 and the program links against libcbessfm and the CUDA runtime (CPU); on
the GPU the program's output equals the Python binding's bit for bit and the FP64 oracle within
the FP32 tolerance, and the documented error paths answer as declared."""
import glob
import os
import shutil
import subprocess

import numpy as np
import pytest

from parity_utils import Case, case_taps, make_plan, oracle_params, random_field, rel_l2, to_storage

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_example.c")


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _cuda_lib_dirs(home):
    dirs = [os.path.join(home, "lib64")] + glob.glob(os.path.join(home, "targets", "*", "lib"))
    return [d for d in dirs if glob.glob(os.path.join(d, "libcudart.so*"))]


def _build_example(out_dir):
    from paper_2409_14489_gb300 import build
    home = _cuda_home()
    libs = _cuda_lib_dirs(home)
    if not libs:
        pytest.skip("no shared CUDA runtime library found")
    exe = os.path.join(out_dir, "c_abi_example")
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(home, "include"), SRC, "-o", exe,
           "-L", os.path.dirname(build.LIB), "-lcbessfm", "-Wl,-rpath," + os.path.dirname(build.LIB)]
    for d in libs:
        cmd += ["-L", d, "-Wl,-rpath," + d]
    cmd += ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_is_c99_and_example_links(tmp_path):
    from paper_2409_14489_gb300 import build
    if not os.path.exists(build.LIB):
        pytest.skip("library not built")
    exe = _build_example(str(tmp_path))
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_program_matches_binding_and_oracle(tmp_path):
    import torch
    from oracle import dbp as odbp
    case = Case(3, 256, 64, 3, 7, 0.3, 3 * 768 + 123, sample_rate=192e9, seed=11)
    taps = case_taps(case).astype(np.float32)
    field = random_field(case)[0].astype(np.complex64)
    exe = _build_example(str(tmp_path))
    fin, ftaps, fout = (str(tmp_path / n) for n in ("in.bin", "taps.bin", "out.bin"))
    field.view(np.float32).tofile(fin)
    taps.tofile(ftaps)
    args = [exe, fin, ftaps, fout, str(case.n_sb), str(case.n_st), str(case.ntaps),
            str(case.n_fft), str(case.overlap), str(case.L), repr(case.ratio), repr(case.beta2),
            repr(case.span_length), str(case.n_spans), repr(case.sample_rate)]
    r = subprocess.run(args, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.fromfile(fout, dtype=np.complex64).reshape(case.L, 2)
    plan = make_plan(case, taps)
    ref = plan.backpropagate(to_storage(field[None].astype(np.complex128), 0))
    torch.cuda.synchronize()
    assert np.array_equal(got, ref[0].cpu().numpy())
    want = odbp.dbp_mode_b(field.astype(np.complex128),
                           oracle_params(case, taps.astype(np.float64)), case.n_fft, case.overlap)
    assert rel_l2(got, want, "c_abi_example") <= 1e-5
