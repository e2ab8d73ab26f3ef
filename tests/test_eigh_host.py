"""The clover force's Hermitian eigen-solver (paper_2411_18511_gb300/csrc/hr_eigh.cuh,
cyclic complex Jacobi) compiled as plain C++ on the host: A = V diag(w) V^+ and
V^+ V = 1 to 1e-13 on random and nearly degenerate 4 x 4 Hermitian matrices.
(The same header runs per site in the exponential clover force on the GPU.)"""

import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2411_18511_gb300", "csrc")

PROGRAM = r"""
#include <complex>
#include <cstdio>
#include <random>
#include "hr_eigh.cuh"
using namespace hr;
using C = std::complex<double>;
int main() {
    std::mt19937_64 g(7);
    std::normal_distribution<double> nd;
    double worst = 0.0, worst_orth = 0.0;
    for (int trial = 0; trial < 3000; ++trial) {
        zd A[4][4], A0[4][4], V[4][4];
        double w[4];
        for (int i = 0; i < 4; ++i)
            for (int j = i; j < 4; ++j) {
                if (i == j) A[i][i] = {2.0 + nd(g), 0.0};
                else { A[i][j] = {nd(g), nd(g)}; A[j][i] = {A[i][j].re, -A[i][j].im}; }
            }
        if (trial % 3 == 0) {  // nearly degenerate
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    if (i != j) { A[i][j].re *= 1e-9; A[i][j].im *= 1e-9; }
            A[1][1] = A[0][0];
        }
        for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) A0[i][j] = A[i][j];
        jacobi_eigh<4>(A, V, w);
        double err = 0.0, nrm = 0.0, orth = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                C s = 0.0, o = 0.0;
                for (int k = 0; k < 4; ++k) {
                    s += C(V[i][k].re, V[i][k].im) * w[k] * std::conj(C(V[j][k].re, V[j][k].im));
                    o += std::conj(C(V[k][i].re, V[k][i].im)) * C(V[k][j].re, V[k][j].im);
                }
                err += std::norm(s - C(A0[i][j].re, A0[i][j].im));
                nrm += std::norm(C(A0[i][j].re, A0[i][j].im));
                orth += std::norm(o - (i == j ? 1.0 : 0.0));
            }
        if (std::sqrt(err / nrm) > worst) worst = std::sqrt(err / nrm);
        if (std::sqrt(orth) > worst_orth) worst_orth = std::sqrt(orth);
    }
    std::printf("%.3e %.3e\n", worst, worst_orth);
    return 0;
}
"""


def test_jacobi_eigh_on_the_host(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "eigh.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "eigh"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    recon, orth = float(out[0]), float(out[1])
    assert recon < 1e-13 and orth < 1e-13, (recon, orth)
