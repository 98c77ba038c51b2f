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


def test_bijection_arithmetic_matches_oracle(orc):
    """The product's integer bijection (host build of csrc/bijection.cuh) gives the oracle's
    pairing positions and inverse for the oracle's round keys, on sizes across the range."""
    import numpy as np
    sizes = [4097, 4098, 5000, 9999, 10000, 12288, 12289, 20000, 32768, 49153, 65535, 65536]
    reqs, refs = [], []
    for i, n in enumerate(sizes):
        fwd, prm = orc.bij_table(1234, 17 * i, 5 + i, n)
        inv, _ = orc.bij_table(1234, 17 * i, 5 + i, n, inverse=True)
        reqs.append(" ".join(str(int(v)) for v in [n, *prm[2:8]]))
        refs.append((int(prm[0]), int(prm[1]), fwd, inv))
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "bijection_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "bijection_check.cpp")],
                       check=True)
        out = subprocess.run([exe], input="\n".join(reqs) + "\n", check=True, capture_output=True,
                             text=True).stdout.splitlines()
    assert out[-1] == "bijection arithmetic OK", out[-1]
    for k, (a, b, fwd, inv) in enumerate(refs):
        ga, gb = (int(v) for v in out[3 * k].split())
        assert (ga, gb) == (a, b)
        assert np.array_equal(np.array(out[3 * k + 1].split(), np.uint32), fwd)
        assert np.array_equal(np.array(out[3 * k + 2].split(), np.uint32), inv)
