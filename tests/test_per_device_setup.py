"""Host-only check of the per-device one-time set-up used before kernel launches
(csrc/per_device.h): the set-up runs once for each device index, again for a new
device, and on every call for an index it cannot remember.  Compiled with the
host C++ compiler; no GPU involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include "per_device.h"
int main() {
  std::atomic<uint64_t> done{0};
  int runs[80] = {};
  const int seq[] = {0, 0, 1, 0, 1, 5, 63, 63, 70, 70, 5};
  for (int d : seq) stm::once_for_device(done, d, [&] { runs[d]++; });
  std::printf("%d %d %d %d %d\n", runs[0], runs[1], runs[5], runs[63], runs[70]);
  return 0;
}
'''


def test_once_for_device(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "t.cc"
    src.write_text(SRC)
    exe = tmp_path / "t"
    subprocess.run([cxx, "-std=c++17", "-I", os.path.join(ROOT, "paper_1307_5310_gb300", "csrc"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out == ["1", "1", "1", "1", "2"]
