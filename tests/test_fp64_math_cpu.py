"""The FP64 helpers of the CUDA path's FP64 mode (csrc/fp64_math.cuh), built
for the host with the same IEEE operations the device runs (fma, add,
multiply and integer bit operations; no contraction):

* widen_f32 returns the conversion instruction's double for every float bit
  pattern below 2^24 (zeros, all subnormals, the smallest normals), every
  subnormal with the sign set, and a stride-7 sweep of all other finite
  patterns;
* exp_tang (Tang's table-driven exponential with a correctly rounded
  2^(j/256) table) is within one unit in the last place of long double exp
  over 2e7 points of [-707, 0], equals 1 at 0 and hands NaN and arguments
  outside its range to the library exp."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fp64_helpers_on_the_host(tmp_path):
    exe = str(tmp_path / "fp64_math_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "paper_1406_5161_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fp64_math_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe, "7"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout
