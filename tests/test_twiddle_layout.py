"""The twiddle array's pass-major tables, checked on the host with the library's own index code
(csrc/fft.cuh compiled by nvcc into a host program; no GPU): every factor a Stockham pass reads
at stk_twp(N, p) + (r - 1) NS + jm is the plain table's entry jm r SWENSE_MAX_FFT / (NS R), the
tables of size N stay inside [SWENSE_MAX_FFT + N, SWENSE_MAX_FFT + 2 N) and no two slots overlap,
and the plain table is the identity. A wrong offset or stride here would feed a transform wrong
twiddles only at the sizes and passes that read the moved entries."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_12716_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

CHECK = r"""
#include <cstdio>
#include <vector>
#include "fft.cuh"
using namespace swense;
int main() {
  long bad = 0, checked = 0;
  std::vector<int> owner(kTwiddleLen, 0);
  for (int j = 0; j < SWENSE_MAX_FFT; ++j) bad += twiddle_exponent(j) != j;
  for (int k = 3; (1 << k) <= SWENSE_MAX_FFT; ++k) {
    const int n = 1 << k;
    for (int p = 1; p < stk_npass(n); ++p) {
      const int ns = stk_ns(n, p), R = stk_radix(n, p);
      for (int r = 1; r < R; ++r)
        for (int jm = 0; jm < ns; ++jm) {
          const int idx = stk_twp(n, p) + (r - 1) * ns + jm;
          ++checked;
          if (idx < SWENSE_MAX_FFT + n || idx >= SWENSE_MAX_FFT + 2 * n || idx >= kTwiddleLen) { ++bad; continue; }
          bad += owner[idx]++ != 0;
          bad += twiddle_exponent(idx) != jm * r * (SWENSE_MAX_FFT / (ns * R));
        }
    }
  }
  std::printf("%ld %ld %d\n", checked, bad, SWENSE_MAX_FFT);
  return bad != 0;
}
"""


def test_pass_major_tables_hold_the_plain_entries(tmp_path):
    from paper_2005_12716_gb300 import build
    try:
        exe = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    src = tmp_path / "twiddle_check.cu"
    src.write_text(CHECK)
    out = tmp_path / "twiddle_check"
    r = subprocess.run([exe, "-std=c++17", "--expt-relaxed-constexpr", *build.ARCH, "-I", INCLUDE,
                        "-I", CSRC, str(src), "-o", str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(out)], capture_output=True, text=True, timeout=60)
    checked, bad, nmax = (int(v) for v in r.stdout.split())
    # every (size, pass, r, jm) of the sizes 8 .. SWENSE_MAX_FFT: N - NS_1 = N - 8 per size
    assert checked == sum((1 << k) - 8 for k in range(3, nmax.bit_length()))
    assert bad == 0 and r.returncode == 0
