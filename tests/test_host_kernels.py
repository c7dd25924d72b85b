"""Host emulation of the shared-memory Stockham FFT used by the CUDA kernels
(paper_2103_01874_gb300/csrc/fft.cuh), against a naive long-double DFT: the
threads of a CTA are run one after another, which is exact for these passes.
Covers every radix (16, 8, 4, 2, 3), both line layouts the kernels use, odd and
radix-3-heavy lengths, both directions, FP32 and FP64."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fft_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if not gxx or not os.path.isdir(inc):
        pytest.skip("g++ or CUDA headers not available")
    exe = str(tmp_path_factory.mktemp("fft") / "fh")
    subprocess.run([gxx, "-O2", "-std=c++20", "-ffp-contract=off", "-I", inc,
                    "-I", os.path.join(ROOT, "paper_2103_01874_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fft_harness.cpp"), "-o", exe], check=True)
    return exe


CASES = []
for n in (8, 9, 12, 16, 18, 24, 27, 32, 48, 64, 96, 128, 192, 256, 384, 512):
    CASES.append(("f", n, 16, 1, 16, 16))          # z / y layout: [e][line], 16 lines
    CASES.append(("d", n, 8, 1, 8, 8))
    CASES.append(("f", n, 8, n + 1, 1, 16))        # x layout: padded lines
CASES.append(("d", 1024, 2, 1025, 1, 8))


CT_SIZES = (16, 24, 32, 48, 64, 96, 128, 192, 256, 384)


@pytest.mark.parametrize("mode", ["runtime", "ct"])
@pytest.mark.parametrize("inv", [0, 1])
@pytest.mark.parametrize("typ,n,nl,ls,es,maxr", CASES)
def test_stockham_matches_dft(fft_exe, typ, n, nl, ls, es, maxr, inv, mode):
    """Both the run-time-length passes and the compile-time-length passes
    (fft_lines_ct, used for the common lengths) against the naive DFT."""
    if mode == "ct" and n not in CT_SIZES:
        pytest.skip("no compile-time instance for this length")
    args = [fft_exe, typ, str(inv), str(n), str(nl), str(ls), str(es), str(maxr)] + (["c"] if mode == "ct" else [])
    out = subprocess.run(args, capture_output=True, text=True, check=True)
    err = float(out.stdout.strip())
    assert 0 <= err < (1e-6 if typ == "f" else 1e-14), err
