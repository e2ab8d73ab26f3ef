"""The clover force's per-link plaquette sum (paper_2411_18511_gb300/csrc/
hr_clover_leaf.cuh, the code the GPU kernel runs per link) compiled as plain
C++ on the host, against the oracle's leaf-by-leaf derivative
(oracle.clover.clover_derivative) for a random insertion: both take the same
K_mn = tr_s[(s_mn (x) 1) Lam]."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth
from oracle import clover as ocl

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2411_18511_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "hr_clover_leaf.cuh"
using namespace hr;
int main(int argc, char **argv) {
    LeafLattice L;
    FILE *f = std::fopen(argv[1], "rb");
    if (std::fread(L.d, sizeof(int), 4, f) != 4) return 1;
    const long long V = (long long)L.d[0] * L.d[1] * L.d[2] * L.d[3];
    std::vector<double> can(16 * V), K(48 * V), F(12 * V);
    if (std::fread(can.data(), sizeof(double), can.size(), f) != can.size()) return 1;
    if (std::fread(K.data(), sizeof(double), K.size(), f) != K.size()) return 1;
    std::fclose(f);
    for (int rho = 0; rho < 4; ++rho)
        for (long long z = 0; z < V; ++z) {
            int x[4];
            long long r = z;
            for (int k = 3; k >= 0; --k) { x[k] = (int)(r % L.d[k]); r /= L.d[k]; }
            double out[3];
            leaf_force_link(L, can.data(), K.data(), rho, x, out);
            for (int a = 0; a < 3; ++a) F[(rho * V + z) * 3 + a] = out[a];
        }
    f = std::fopen(argv[2], "wb");
    std::fwrite(F.data(), sizeof(double), F.size(), f);
    std::fclose(f);
    return 0;
}
"""

PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 2, 4, 2), (4, 4, 2, 6)])
def test_plaquette_sum_matches_leaf_by_leaf(tmp_path, dims):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "leaf"
    src = tmp_path / "leaf.cpp"
    src.write_text(PROGRAM)
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    V = int(np.prod(dims))
    rng = np.random.default_rng(701)
    q = synth.haar_links(dims, 702)
    Lam = rng.normal(size=(V, 8, 8)) + 1j * rng.normal(size=(V, 8, 8))
    L4 = Lam.reshape(V, 4, 2, 4, 2)
    K = np.stack([np.einsum("st,xtbsa->xba", ocl.sigma(mu, nu), L4) for mu, nu in PLANES], axis=1)  # [V,6,2,2]
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as fh:
        fh.write(np.asarray(dims, dtype=np.int32).tobytes())
        fh.write(np.ascontiguousarray(q, dtype=np.float64).tobytes())
        fh.write(np.ascontiguousarray(K, dtype=np.complex128).tobytes())
    out = tmp_path / "out.bin"
    subprocess.run([str(exe), str(inp), str(out)], check=True)
    F = np.fromfile(out, dtype=np.float64).reshape(4, V, 3)
    want = ocl.clover_derivative(dims, oracle.expand_links(dims, 2, q), Lam)
    assert np.linalg.norm(F - want) <= 1e-13 * np.linalg.norm(want)
