"""The integer-pipe double product of the kernels (csrc/fv_emu.h), compiled
for the host and checked bit for bit against the host's IEEE-754
multiplication on 4e6 operand pairs: ordinary products, short significands
(exact products and ties to even), results at the edges of the normal range,
zeros, subnormals, infinities and NaN, and significands whose rounding carries
into the exponent.  The same source runs in the GPU kernels; on the GPU it is
checked against the FP64 multiplier (tests/test_gpu_bits.py)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_pipe_product_equals_ieee_multiplication(tmp_path):
    exe = str(tmp_path / "emu_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-Wall", "-o", exe,
                    os.path.join(HERE, "native", "emu_check.cpp")], check=True)
    p = subprocess.run([exe, "4000000"], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    cases, fast, bad = (int(x) for x in p.stdout.split()[-3:])
    assert cases == 4000000 and bad == 0
    assert fast > 0.5 * cases  # most pairs take the integer path
