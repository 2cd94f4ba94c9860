"""The small dense algebra of the GPU GCRO-DR (csrc/gcro_small.cuh), compiled
for the host and checked against numpy / scipy on the CPU:

* eigen-decomposition (Hessenberg reduction + complex QR with Wilkinson
  shifts + Schur eigenvectors) of random complex matrices: eigenvalues equal
  numpy's, and every M x = lambda x holds to 1e-10;
* Householder least squares equals numpy.linalg.lstsq;
* the seed driver (a GMRES cycle that seeds the recycle space) and the cycle
  driver (a cycle with a recycle space) against the same formulas written
  with numpy / scipy: the correction y, and the spans of the new recycle
  coefficients (the harmonic Ritz vectors of smallest modulus are unique up
  to scaling, so C = W Q and U = V^ P R^{-1} are compared as subspaces).
"""
import os
import shutil
import subprocess
import textwrap

import numpy as np
import pytest
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2211_13719_gb300", "csrc", "gcro_small.cuh")

PROGRAM = textwrap.dedent(r"""
    #include <cstdio>
    #include <cstring>
    #include <vector>
    #include "gcro_small.cuh"
    using namespace mrhs::gcro;
    static void rd(std::vector<zc> &M, int rows, int cols) {
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < cols; ++j) { double a, b; if (scanf("%lf %lf", &a, &b) != 2) return; M[i * LD + j] = zc{a, b}; }
    }
    static void wr(const std::vector<zc> &M, int rows, int cols) {
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < cols; ++j) printf("%.17g %.17g\n", M[i * LD + j].re, M[i * LD + j].im);
    }
    int main() {
        char op[16];
        std::vector<zc> ws((size_t)GCRO_WS * LD * LD);
        while (scanf("%15s", op) == 1) {
            if (!strcmp(op, "eig")) {
                int n; scanf("%d", &n);
                std::vector<zc> M(LD * LD), X(LD * LD), Z(LD * LD), lam(LD);
                rd(M, n, n);
                int ok = eig(M.data(), n, lam.data(), X.data(), Z.data());
                printf("%d\n", ok); wr(lam, 1, n); wr(X, n, n);
            } else if (!strcmp(op, "lstsq")) {
                int r, c; scanf("%d %d", &r, &c);
                std::vector<zc> A(LD * LD), b(LD), y(LD);
                rd(A, r, c);
                for (int i = 0; i < r; ++i) { double a, bb; scanf("%lf %lf", &a, &bb); b[i] = zc{a, bb}; }
                lstsq(A.data(), b.data(), r, c, y.data());
                wr(y, 1, c);
            } else if (!strcmp(op, "seed")) {
                int m, k; double beta; scanf("%d %d %lf", &m, &k, &beta);
                std::vector<zc> H(LD * LD), y(LD), qc(LD * LD), pu(LD * LD);
                rd(H, m + 1, m);
                int ok = gcro_seed(H.data(), beta, m, k, y.data(), qc.data(), pu.data(), ws.data());
                printf("%d\n", ok); wr(y, 1, m); wr(qc, m + 1, k); wr(pu, m, k);
            } else if (!strcmp(op, "cycle")) {
                int m, k; scanf("%d %d", &m, &k);
                const int p = m - k;
                std::vector<zc> H(LD * LD), B(LD * LD), wr_(LD), wu(LD * LD), y(LD), qc(LD * LD), pu(LD * LD);
                std::vector<double> un2(LD);
                rd(H, p + 1, p); rd(B, k, p);
                for (int i = 0; i < k; ++i) scanf("%lf", &un2[i]);
                for (int i = 0; i <= m; ++i) { double a, b; scanf("%lf %lf", &a, &b); wr_[i] = zc{a, b}; }
                rd(wu, m + 1, k);
                int ok = gcro_cycle(H.data(), B.data(), un2.data(), wr_.data(), wu.data(), m, k, y.data(), qc.data(),
                                    pu.data(), ws.data());
                printf("%d\n", ok); wr(y, 1, m); wr(qc, m + 1, k); wr(pu, m, k);
            }
            fflush(stdout);
        }
        return 0;
    }
""")


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("gcro")
    src = d / "gcro_small_host.cpp"
    src.write_text(PROGRAM)
    exe = d / "gcro_small_host"
    subprocess.run([cxx, "-std=c++17", "-O2", "-w", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(prog, text):
    return subprocess.run([prog], input=text, capture_output=True, text=True, check=True).stdout.split()


def _fmt(M):
    return "\n".join(f"{float(z.real)!r} {float(z.imag)!r}" for z in np.asarray(M, complex).ravel())


def _read(tok, pos, rows, cols):
    vals = np.array([float(t) for t in tok[pos:pos + 2 * rows * cols]])
    return (vals[0::2] + 1j * vals[1::2]).reshape(rows, cols), pos + 2 * rows * cols


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _span_dist(A, B):
    """sine of the largest principal angle between span(A) and span(B): the norm
    of the part of an orthonormal basis of span(B) outside span(A)."""
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    return float(np.linalg.norm(qb - qa @ (qa.conj().T @ qb), 2))


@pytest.mark.parametrize("n", [3, 8, 14, 16])
def test_eig_matches_numpy(prog, n):
    rng = np.random.default_rng(n)
    M = _rand(rng, n, n)
    tok = _run(prog, f"eig {n}\n{_fmt(M)}\n")
    assert tok[0] == "1"
    lam, pos = _read(tok, 1, 1, n)
    X, _ = _read(tok, pos, n, n)
    lam = lam[0]
    ref = np.linalg.eigvals(M)
    assert np.abs(np.sort_complex(lam) - np.sort_complex(ref)).max() < 1e-10 * np.abs(ref).max()
    for s in range(n):
        x = X[:, s]
        assert np.linalg.norm(M @ x - lam[s] * x) <= 1e-10 * np.linalg.norm(M) * np.linalg.norm(x)


def test_lstsq_matches_numpy(prog):
    rng = np.random.default_rng(5)
    A, b = _rand(rng, 15, 14), _rand(rng, 15)
    tok = _run(prog, f"lstsq 15 14\n{_fmt(A)}\n{_fmt(b)}\n")
    y, _ = _read(tok, 0, 1, 14)
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.abs(y[0] - ref).max() < 1e-12 * np.abs(ref).max()


def _arnoldi(A, r, steps):
    N = len(r)
    V = np.zeros((N, steps + 1), complex)
    H = np.zeros((steps + 1, steps), complex)
    V[:, 0] = r / np.linalg.norm(r)
    for j in range(steps):
        w = A @ V[:, j]
        for i in range(j + 1):
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


def test_seed_driver_matches_formulas(prog):
    rng = np.random.default_rng(11)
    N, m, k = 40, 10, 3
    A = _rand(rng, N, N) + 8 * np.eye(N)
    r = _rand(rng, N)
    V, H = _arnoldi(A, r, m)
    beta = np.linalg.norm(r)
    tok = _run(prog, f"seed {m} {k} {float(beta)!r}\n{_fmt(H)}\n")
    assert tok[0] == "1"
    y, pos = _read(tok, 1, 1, m)
    qc, pos = _read(tok, pos, m + 1, k)
    pu, _ = _read(tok, pos, m, k)
    e1 = np.zeros(m + 1, complex)
    e1[0] = beta
    assert np.abs(y[0] - np.linalg.lstsq(H, e1, rcond=None)[0]).max() < 1e-10
    # harmonic Ritz vectors of smallest modulus, written directly
    Hm = H[:m]
    em = np.zeros(m)
    em[-1] = 1
    F = Hm + abs(H[m, m - 1]) ** 2 * np.outer(np.linalg.solve(Hm.conj().T, em), em)
    th, Z = np.linalg.eig(F)
    P = Z[:, np.argsort(np.abs(th), kind="stable")[:k]]
    Q, R = np.linalg.qr(H @ P)
    U_ref, C_ref = V[:, :m] @ P @ np.linalg.inv(R), V @ Q
    U, Cn = V[:, :m] @ pu, V @ qc
    assert _span_dist(U, U_ref) < 1e-8 and _span_dist(Cn, C_ref) < 1e-8
    assert np.abs(A @ U - Cn).max() < 1e-8 * np.abs(Cn).max()      # C = A U
    assert np.abs(Cn.conj().T @ Cn - np.eye(k)).max() < 1e-10        # orthonormal


def test_cycle_driver_matches_formulas(prog):
    rng = np.random.default_rng(12)
    N, m, k = 48, 10, 3
    p = m - k
    A = _rand(rng, N, N) + 8 * np.eye(N)
    # a recycle space with C = A U orthonormal
    U0 = _rand(rng, N, k)
    C, Rc = np.linalg.qr(A @ U0)
    U = U0 @ np.linalg.inv(Rc) * np.array([1.7, 0.6, 2.3])           # columns of different norm
    C = A @ U
    C, Rc = np.linalg.qr(C)
    U = U @ np.linalg.inv(Rc)
    # a residual orthogonal to C, as GCRO-DR keeps it (x += U C^H r makes r -= C C^H r)
    r = _rand(rng, N)
    r = r - C @ (C.conj().T @ r)
    # Arnoldi of (I - C C^H) A from r
    V = np.zeros((N, p + 1), complex)
    H = np.zeros((p + 1, p), complex)
    B = np.zeros((k, p), complex)
    V[:, 0] = r / np.linalg.norm(r)
    for j in range(p):
        w = A @ V[:, j]
        B[:, j] = C.conj().T @ w
        w = w - C @ B[:, j]
        for i in range(j + 1):
            H[i, j] = np.vdot(V[:, i], w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    W = np.concatenate([C, V], axis=1)
    un2 = np.sum(np.abs(U) ** 2, axis=0)
    wr = W.conj().T @ r
    wu = W.conj().T @ U
    text = f"cycle {m} {k}\n{_fmt(H)}\n{_fmt(B)}\n" + "\n".join(repr(float(x)) for x in un2) + f"\n{_fmt(wr)}\n{_fmt(wu)}\n"
    tok = _run(prog, text)
    assert tok[0] == "1"
    y, pos = _read(tok, 1, 1, m)
    qc, pos = _read(tok, pos, m + 1, k)
    pu, _ = _read(tok, pos, m, k)
    dn = 1 / np.sqrt(un2)
    G = np.zeros((m + 1, m), complex)
    G[:k, :k] = np.diag(dn)
    G[:k, k:] = B
    G[k:, k:] = H
    Vh = np.concatenate([U * dn[None, :], V[:, :p]], axis=1)
    y_ref = np.linalg.lstsq(G, W.conj().T @ r, rcond=None)[0]
    x_corr = U @ y[0][:k] + V[:, :p] @ y[0][k:]
    assert np.abs(x_corr - Vh @ y_ref).max() < 1e-9 * np.abs(Vh @ y_ref).max()
    th, Z = scipy.linalg.eig(G.conj().T @ G, G.conj().T @ (W.conj().T @ Vh))
    mod = np.where(np.isfinite(th), np.abs(th), np.inf)
    P = Z[:, np.argsort(mod, kind="stable")[:k]]
    Q, R = np.linalg.qr(G @ P)
    C_ref, U_ref = W @ Q, Vh @ P @ np.linalg.inv(R)
    Cn = C @ qc[:k] + V @ qc[k:]
    Un = U @ pu[:k] + V[:, :p] @ pu[k:]
    assert _span_dist(Cn, C_ref) < 1e-8 and _span_dist(Un, U_ref) < 1e-8
    assert np.abs(A @ Un - Cn).max() < 1e-8 * np.abs(Cn).max()
