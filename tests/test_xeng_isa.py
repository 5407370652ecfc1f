"""The instruction-set fact behind the X-engine's tensor-core form: on sm_103a
the 8-bit integer kind of the fifth-generation tensor-core MMA
(tcgen05.mma kind::i8) is refused by ptxas, while the same source assembles
for sm_100a; the FP8 kind (kind::f8f6f4) that the X-engine uses assembles for
sm_103a.  CPU only (nvcc cross-compiles)."""
import os
import shutil
import subprocess
import tempfile

import pytest

SRC = r"""
#include <cstdint>
__global__ void k(uint32_t d, uint64_t a, uint64_t b, uint32_t id) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n\t}"
               :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(1));
}
"""


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not available")


def _assemble(kind, arch):
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "k.cu")
        open(src, "w").write(SRC.replace("KIND", kind))
        r = subprocess.run([_nvcc(), "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", src,
                            "-o", os.path.join(d, "k.o")], capture_output=True, text=True)
        return r.returncode, r.stdout + r.stderr


def test_kind_i8_refused_on_sm103a():
    rc, out = _assemble("i8", "103a")
    assert rc != 0 and "not supported on .target 'sm_103a'" in out
    rc100, out100 = _assemble("i8", "100a")
    assert rc100 == 0, out100


def test_kind_f8f6f4_assembles_on_sm103a():
    rc, out = _assemble("f8f6f4", "103a")
    assert rc == 0, out
