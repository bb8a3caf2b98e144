// Host-side set-up of the fast-diagonalisation solver (FP64, runs once per handle).
//
// The paper's Remark after Algorithm 2 notes that every linear system of the
// step has a constant coefficient matrix that can be pre-computed.  On the
// tensor-product mesh each of those matrices is
//     A = Kx (x) My + Mx (x) Ky + c Mx (x) My
// (GLL quadrature makes the mass diagonal and the stiffness separable), so one
// generalised eigendecomposition per direction and boundary-condition set
// diagonalises all of them:  K s = lambda M s,  s^T M s = 1.
//
// This file builds the GLL tables (Sec. 3.2.1 element basis), the assembled 1D
// stiffness and mass of a row of elements, and the eigenbasis (symmetric
// Jacobi rotations on M^{-1/2} K M^{-1/2}).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/pf.h"

namespace {

// Legendre P_K and its first derivative at x by the three-term recurrence.
void legendre(int K, double x, double &p, double &dp) {
    double p0 = 1.0, p1 = x;
    if (K == 0) { p = 1.0; dp = 0.0; return; }
    for (int k = 2; k <= K; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    p = p1;
    // (1 - x^2) P_K' = K (P_{K-1} - x P_K)
    dp = (std::fabs(1.0 - x * x) > 0.0) ? K * (p0 - x * p1) / (1.0 - x * x) : 0.0;
}

}  // namespace

extern "C" int pf_gll(int K, double *nodes, double *weights, double *D) {
    if (K < 1 || K > 31 || !nodes || !weights || !D) return PF_EINVAL;
    const int n = K + 1;
    nodes[0] = -1.0;
    nodes[K] = 1.0;
    // interior nodes: roots of P_K', Newton from the Chebyshev-Gauss-Lobatto points;
    // P_K'' comes from Legendre's equation (1-x^2) P'' = 2 x P' - K (K+1) P.
    for (int j = 1; j < K; ++j) {
        double x = -std::cos(M_PI * j / K);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(K, x, p, dp);
            double ddp = (2.0 * x * dp - K * (K + 1.0) * p) / (1.0 - x * x);
            double dx = dp / ddp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        nodes[j] = x;
    }
    std::vector<double> pk(n);
    for (int j = 0; j < n; ++j) {
        double p, dp;
        legendre(K, nodes[j], p, dp);
        pk[j] = p;
        weights[j] = 2.0 / (K * (K + 1.0) * p * p);
    }
    // closed-form GLL differentiation matrix
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            if (i != j) v = pk[i] / (pk[j] * (nodes[i] - nodes[j]));
            else if (i == 0) v = -0.25 * K * (K + 1.0);
            else if (i == K) v = 0.25 * K * (K + 1.0);
            D[i * n + j] = v;
        }
    return PF_OK;
}

extern "C" int pf_nodes_1d(int ne, const double *br, int K, int periodic, double *nodes) {
    if (ne < 1 || K < 1 || K > 31 || !br || !nodes) return PF_EINVAL;
    for (int e = 0; e < ne; ++e)
        if (!(br[e + 1] > br[e])) return PF_EINVAL;
    std::vector<double> x(K + 1), w(K + 1), D((K + 1) * (K + 1));
    pf_gll(K, x.data(), w.data(), D.data());
    for (int e = 0; e < ne; ++e)
        for (int a = 0; a < K; ++a) nodes[e * K + a] = br[e] + 0.5 * (x[a] + 1.0) * (br[e + 1] - br[e]);
    if (!periodic) nodes[ne * K] = br[ne];
    return PF_OK;
}

extern "C" int pf_operators_1d(int ne, const double *br, int K, int periodic, double *Kmat,
                               double *Mdiag) {
    if (ne < 1 || K < 1 || K > 31 || !br || !Kmat || !Mdiag) return PF_EINVAL;
    for (int e = 0; e < ne; ++e)
        if (!(br[e + 1] > br[e])) return PF_EINVAL;
    const int p = K + 1;
    const int n = periodic ? ne * K : ne * K + 1;
    if (periodic && n < 2) return PF_EINVAL;
    std::vector<double> x(p), w(p), D(p * p);
    pf_gll(K, x.data(), w.data(), D.data());
    std::fill(Kmat, Kmat + (size_t)n * n, 0.0);
    std::fill(Mdiag, Mdiag + n, 0.0);
    for (int e = 0; e < ne; ++e) {
        const double h = br[e + 1] - br[e];
        for (int a = 0; a < p; ++a) {
            const int ga = (e * K + a) % n;
            Mdiag[ga] += 0.5 * h * w[a];
            for (int c = 0; c < p; ++c) {
                const int gc = (e * K + c) % n;
                double s = 0.0;
                for (int q = 0; q < p; ++q) s += w[q] * D[q * p + a] * D[q * p + c];
                Kmat[(size_t)ga * n + gc] += (2.0 / h) * s;
            }
        }
    }
    return PF_OK;
}

namespace {

// Symmetric eigendecomposition by cyclic Jacobi rotations: A = V diag(ev) V^T.
// A is m x m row-major and is destroyed.  A rotation is skipped once
// |a_pq| <= 1e-17 sqrt(|a_pp a_qq|) (negligible relative to the diagonal) or below an
// absolute floor 1e-22 ||A||_F; the sweeps stop when a sweep rotates nothing.  The relative
// test keeps rotating until the small eigenvalues are resolved to relative accuracy,
// which the fast-diagonalisation solves of the Laplace-type (c = 0) systems need.
void jacobi_eig(int m, std::vector<double> &A, std::vector<double> &V, std::vector<double> &ev) {
    V.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
    double fro = 0.0;
    for (size_t i = 0; i < A.size(); ++i) fro += A[i] * A[i];
    fro = std::sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < m - 1; ++p) {
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[(size_t)p * m + q];
                const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                if (std::fabs(apq) <= 1e-17 * std::sqrt(std::fabs(app * aqq)) || std::fabs(apq) <= 1e-22 * fro) {
                    continue;
                }
                ++rotated;
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                // columns p, q
                for (int k = 0; k < m; ++k) {
                    double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
                    A[(size_t)k * m + p] = c * akp - s * akq;
                    A[(size_t)k * m + q] = s * akp + c * akq;
                }
                // rows p, q
                for (int k = 0; k < m; ++k) {
                    double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
                    A[(size_t)p * m + k] = c * apk - s * aqk;
                    A[(size_t)q * m + k] = s * apk + c * aqk;
                }
                A[(size_t)p * m + q] = 0.0;
                A[(size_t)q * m + p] = 0.0;
                for (int k = 0; k < m; ++k) {
                    double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
                    V[(size_t)k * m + p] = c * vkp - s * vkq;
                    V[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
        }
        if (!rotated) break;
    }
    ev.resize(m);
    for (int i = 0; i < m; ++i) ev[i] = A[(size_t)i * m + i];
}

}  // namespace

extern "C" int pf_fdm_1d(int n, const double *Kmat, const double *Mdiag, const unsigned char *dirichlet,
                         double *S, double *lam) {
    if (n < 1 || !Kmat || !Mdiag || !S || !lam) return PF_EINVAL;
    std::vector<int> fr;
    for (int i = 0; i < n; ++i) {
        if (!(Mdiag[i] > 0.0)) return PF_EINVAL;
        if (!dirichlet || !dirichlet[i]) fr.push_back(i);
    }
    const int m = (int)fr.size();
    std::fill(S, S + (size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) lam[i] = 1.0;
    if (m == 0) return PF_OK;
    std::vector<double> A((size_t)m * m), V, ev;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            A[(size_t)i * m + j] = Kmat[(size_t)fr[i] * n + fr[j]] / std::sqrt(Mdiag[fr[i]] * Mdiag[fr[j]]);
    jacobi_eig(m, A, V, ev);
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    for (int c = 0; c < m; ++c) {
        const int src = ord[c];
        lam[c] = ev[src];
        // fix the sign so that the largest-magnitude entry is positive (deterministic basis)
        double big = 0.0;
        for (int i = 0; i < m; ++i)
            if (std::fabs(V[(size_t)i * m + src]) > std::fabs(big)) big = V[(size_t)i * m + src];
        const double sg = big < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < m; ++i)
            S[(size_t)fr[i] * n + c] = sg * V[(size_t)i * m + src] / std::sqrt(Mdiag[fr[i]]);
    }
    return PF_OK;
}
