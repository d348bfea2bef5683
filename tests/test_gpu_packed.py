"""The packed FP32x2 double-float arithmetic (PrecDF in kg_arith.cuh) against the scalar
double-float forms it replaced, on the GPU: sums, differences, renormalisation, the sqrt(1/2)
rotations of a radix-8 DFT, a + i b, -i a, power-of-two scaling and lam x^3 must give bitwise
the scalar results (each lane runs the same round-to-nearest operations); a twiddle product
bitwise in its real lane, and in its imaginary lane, whose low-order terms are added in another
order, within 1e-13 of the operands' size.  2^20 seeded operand pairs per case, magnitudes
2^-40 .. 2^40 with zeros and unnormalised low words (tests/packed_arith_check.cu)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1501_04552_gb300", "csrc")


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("packed") / "packed_arith_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC,
                    "-o", exe, os.path.join(HERE, "packed_arith_check.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.split("\n"):
        parts = line.split()
        if len(parts) == 4:
            res[parts[0]] = (int(parts[1]), int(parts[2]), float(parts[3]))
    print(out)
    return res


BITWISE = ["cadd", "csub", "cnorm", "crot_plus", "crot_minus", "cadd_i", "cmul_negi_scale", "ccube", "cscale2"]


@pytest.mark.parametrize("case", BITWISE)
def test_packed_forms_are_bitwise_the_scalar_ones(results, case):
    n, mism, rel = results[case]
    assert n == 1 << 20
    assert mism == 0, (case, mism, rel)
    assert rel == 0.0


def test_packed_twiddle_product(results):
    n, mism, rel = results["ctw"]
    assert n == 1 << 20
    assert mism == 0          # the real lane: the same operations in the same order
    assert rel <= 1e-13       # the imaginary lane: the same terms, low-order sum reordered
