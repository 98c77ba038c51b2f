"""Host-side check of the cell kernel's ownership arithmetic (no GPU needed)."""
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cluster_index_arithmetic():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "index_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "index_check.cpp")], check=True)
        out = subprocess.run([exe, "70000"], check=True, capture_output=True, text=True).stdout
        assert "index arithmetic OK" in out, out
