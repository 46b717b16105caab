"""Host logic of the all-assignment kernel, checked on the CPU: the division
by invariant integers used for version indices (exhaustive over its whole
dividend range for the divisors that occur) and the table geometry (regions
disjoint, inside the table, aligned for vector access).  The header is
compiled as host code by nvcc; no GPU is needed."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2502_07060_gb300", "csrc")

PROGRAM = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "bg_states.cuh"
using namespace bgk;

static int fail(const char* what, long a, long b) { printf("FAIL %s %ld %ld\n", what, a, b); return 1; }

int main() {
    // divisors that occur: S (2..255) and S^L <= 2^20; dividends < 2^24
    for (uint32_t d = 1; d <= 255; ++d) {
        for (uint64_t dl = d; dl <= (1u << 20); dl *= d) {
            const DivU q = make_divu((uint32_t)dl);
            const uint32_t step = dl <= 255 || dl == 1024 ? 1 : 977;   // exhaustive for S and one S^L
            for (uint32_t x = 0; x < (1u << 24); x += step)
                if (q.div(x) != x / dl) return fail("div", x, (long)dl);
            for (uint32_t k = 1; k * dl < (1u << 24); k = k * 2 + 1) {   // edges of the quotient steps
                const uint32_t xs[3] = {(uint32_t)(k * dl - 1), (uint32_t)(k * dl), (uint32_t)(k * dl + dl - 1)};
                for (uint32_t x : xs)
                    if (x < (1u << 24) && q.div(x) != x / dl) return fail("div-edge", x, (long)dl);
            }
            if (d == 1) break;
        }
    }
    // geometry: uniform S for every n with S^n * n <= 2^20, and mixed
    // per-leg state counts; every (D, D_s) and element size
    const int dims[6][2] = {{4, 4}, {4, 6}, {4, 8}, {6, 6}, {6, 8}, {8, 8}};
    const int elems[3][2] = {{4, 4}, {16, 16}, {16, 8}};
    int checked = 0;
    std::vector<std::vector<int>> radices;
    for (int n = 4; n <= 12; ++n) {
        for (int S = 1; S <= 255; ++S) {
            long h = 1;
            for (int l = 0; l < n; ++l) h *= S;
            if (h * n > (1 << 20)) break;
            radices.push_back(std::vector<int>(n, S));
        }
        std::vector<int> cut(n, 1);
        cut[0] = cut[n - 1] = 6;
        radices.push_back(cut);
        std::vector<int> mixed(n);
        for (int l = 0; l < n; ++l) mixed[l] = 1 + (l * 7 + 3) % 3;      // 1..3
        long h = 1;
        for (int r : mixed) h *= r;
        if (h * n <= (1 << 20)) radices.push_back(mixed);
    }
    for (const auto& rad : radices) {
        const int n = (int)rad.size();
        int S = 1;
        long H = 1;
        for (int r : rad) { S = r > S ? r : S; H *= r; }
        for (auto& dd : dims)
            for (auto& ee : elems) {
                const int D = dd[0], DS = dd[1];
                const StatesGeometry g = make_states_geometry(n, S, rad.data(), D, DS, ee[0], ee[1]);
                const int N = n - 1;
                if (g.H != H) return fail("H", n, g.H);
                long end = 0;                          // regions in order, contiguous
                for (int L = 1; L < N; ++L)
                    for (int i = 0; i + L <= N; ++i) {
                        long w = 1;
                        for (int l = i; l < i + L; ++l) w *= rad[l];
                        if (g.W[i][L] != w) return fail("W", i, L);
                        if (g.cur[L][i] != end || g.cur[L][i] % 2) return fail("cur", L, i);
                        end += w * DS;
                    }
                for (int L = 2; L < N; ++L)
                    for (int i = 0; i + L <= N; ++i) {
                        if (g.sa[L][i] < end) return fail("sa", L, i);
                        end = g.sa[L][i] + g.W[i][L];
                    }
                if (g.off_inv < end || g.off_inv % 4) return fail("inv", n, S);
                int ns = 0;                            // internal ranges: lengths 2..N-1
                for (int L = 2; L < N; ++L) {
                    if (g.inv[L] != ns) return fail("inv-offset", n, L);
                    ns += N - L + 1;
                }
                if (g.ns != ns) return fail("ns", n, g.ns);
                if (g.off_el < g.off_inv + g.ns || g.off_el % 4) return fail("el", n, S);
                if (g.off_k < g.off_el + rad[N] * DS || g.off_k % 4) return fail("k", n, S);
                if ((long)g.off_flag * ee[0] < (long)g.off_k * ee[0] + (long)(N + 1) * D * ee[1])
                    return fail("k-size", n, S);
                if (g.off_flag % 4 || g.words < g.off_flag + 1 || g.words % 4) return fail("words", n, g.words);
                for (int m = 2; m <= N; ++m) {
                    long c = 0;
                    for (int i = 0; i + m <= N; ++i) {
                        if (g.first[m][i] != c) return fail("first", m, i);
                        c += g.W[i][m];
                    }
                    if (g.first[m][N - m + 1] != c || g.count[m] != c) return fail("count", m, c);
                    if ((long)g.P * c >= (1L << 24)) return fail("dividend", m, c);
                    for (long x = 0; x < (long)g.P * c; x += 1 + c / 64)
                        if (g.div_count[m].div((uint32_t)x) != x / c) return fail("div_count", m, x);
                }
                if (g.P < 1 || g.P > 32 || (g.P > 1 && g.P * g.count[N] > 32)) return fail("P", n, g.P);
                ++checked;
            }
    }
    printf("OK %d\n", checked);
    return 0;
}
'''


def test_states_division_and_geometry(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "states_host.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "states_host"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
