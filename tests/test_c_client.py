"""The C ABI from plain C: tests/c_client.c includes only include/ihist.h and
the CUDA runtime's C header, links libihist.so, and drives a plan, a query
and a batch with raw device pointers.  On the CPU it must compile and link
(the header is valid C11 and every symbol it uses is exported); on the GPU
its results must equal the oracle's word for word."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1711_01919_gb300 import build as cuda_build
from paper_1711_01919_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def compile_client(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime_api.h")):
        pytest.skip("no C compiler or CUDA headers")
    lib = cuda_build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_client")
    cmd = [cc, "-std=c11", "-O1", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(cuda_build.ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(HERE, "c_client.c"), "-o", exe,
           "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir,
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.access(compile_client(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_c_client_results_equal_the_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = compile_client(tmp_path)
    h, w, nbins, nrects = 270, 533, 24, 300
    img = synth.gradient_frame(4242, h, w)
    rects = synth.rects(4243, nrects, h, w)
    f_in, f_rects = tmp_path / "frame.u8", tmp_path / "rects.i32"
    f_hist, f_rows = tmp_path / "hist.u32", tmp_path / "rows.u32"
    img.tofile(f_in)
    np.ascontiguousarray(rects, dtype=np.int32).tofile(f_rects)
    r = subprocess.run([exe, str(h), str(w), str(nbins), str(f_in), str(f_rects), str(nrects), str(f_hist),
                        str(f_rows)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c client ok" in r.stdout
    ref = oracle.integral_histogram(img, nbins)
    got = np.fromfile(f_hist, dtype=np.uint32).reshape(nbins, h, w)
    assert np.array_equal(got, ref)
    rows = np.fromfile(f_rows, dtype=np.uint32).reshape(nrects, nbins)
    assert np.array_equal(rows, oracle.query(ref, rects))
