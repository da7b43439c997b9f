// Reference-element tables for the GPU discretisation.
//
// V_h (Sec. 3, the DG space) is represented on each element by the L2-orthonormal
// Dubiner (collapsed-Jacobi) basis of P_p on the unit simplex, pushed forward by the
// affine element map and scaled by 1/sqrt|det J|, so the element mass matrix is the
// identity.  This is what makes the mass solve of Sec. 4 a pointwise 6x6 (3x3 in 2D)
// solve per coefficient ("inversion of a diagonal mass matrix" for straight elements).
//
// Every basis function is expanded exactly into monomials x^a y^b z^c (long double
// arithmetic); every reference integral below is then evaluated by the monomial
// formula  int_{unit d-simplex} x^a y^b z^c = a! b! c! / (a+b+c+d)!,  so the tables
// carry no quadrature error.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "mtp_internal.h"

namespace mtp {
namespace {

typedef long double ld;
constexpr int D = 12;  // degrees up to 11 = 2p + 1 for p = 5

struct Poly {
    ld c[D][D][D];
    Poly() { std::memset(c, 0, sizeof(c)); }
    static Poly cst(ld v) { Poly p; p.c[0][0][0] = v; return p; }
    static Poly var(int i) {
        Poly p;
        if (i == 0) p.c[1][0][0] = 1; else if (i == 1) p.c[0][1][0] = 1; else p.c[0][0][1] = 1;
        return p;
    }
};

Poly add(const Poly& a, const Poly& b, ld sb = 1) {
    Poly r;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            for (int k = 0; k < D; ++k) r.c[i][j][k] = a.c[i][j][k] + sb * b.c[i][j][k];
    return r;
}
Poly scale(const Poly& a, ld s) {
    Poly r;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            for (int k = 0; k < D; ++k) r.c[i][j][k] = s * a.c[i][j][k];
    return r;
}
Poly mul(const Poly& a, const Poly& b) {
    Poly r;
    for (int i = 0; i < D; ++i)
        for (int j = 0; i + j < D; ++j)
            for (int k = 0; i + j + k < D; ++k) {
                ld av = a.c[i][j][k];
                if (av == 0) continue;
                for (int u = 0; u < D; ++u)
                    for (int v = 0; u + v < D; ++v)
                        for (int w = 0; u + v + w < D; ++w) {
                            ld bv = b.c[u][v][w];
                            if (bv == 0) continue;
                            if (i + j + k + u + v + w >= D) throw std::runtime_error("poly degree overflow");
                            r.c[i + u][j + v][k + w] += av * bv;
                        }
            }
    return r;
}
Poly deriv(const Poly& a, int var) {
    Poly r;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            for (int k = 0; k < D; ++k) {
                ld v = a.c[i][j][k];
                if (v == 0) continue;
                if (var == 0 && i > 0) r.c[i - 1][j][k] += v * i;
                if (var == 1 && j > 0) r.c[i][j - 1][k] += v * j;
                if (var == 2 && k > 0) r.c[i][j][k - 1] += v * k;
            }
    return r;
}
ld fact(int n) { ld r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
// integral over the unit simplex of dimension d (variables x[, y[, z]])
ld integrate(const Poly& a, int d) {
    ld s = 0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            for (int k = 0; k < D; ++k) {
                ld v = a.c[i][j][k];
                if (v == 0) continue;
                if ((d < 3 && k > 0) || (d < 2 && j > 0)) throw std::runtime_error("variable outside simplex dim");
                s += v * fact(i) * fact(j) * fact(k) / fact(i + j + k + d);
            }
    return s;
}
ld eval(const Poly& a, ld x, ld y, ld z) {
    ld s = 0, xi = 1;
    for (int i = 0; i < D; ++i, xi *= x) {
        ld yj = 1;
        for (int j = 0; j < D; ++j, yj *= y) {
            ld zk = 1;
            for (int k = 0; k < D; ++k, zk *= z) s += a.c[i][j][k] * xi * yj * zk;
        }
    }
    return s;
}
// a(X(s), Y(s), Z(s)) for polynomial substitutions X, Y, Z
Poly compose(const Poly& a, const Poly& X, const Poly& Y, const Poly& Z) {
    Poly Xp[D], Yp[D], Zp[D];
    Xp[0] = Yp[0] = Zp[0] = Poly::cst(1);
    for (int i = 1; i < D; ++i) { Xp[i] = mul(Xp[i - 1], X); Yp[i] = mul(Yp[i - 1], Y); Zp[i] = mul(Zp[i - 1], Z); }
    Poly r;
    for (int i = 0; i < D; ++i)
        for (int j = 0; i + j < D; ++j)
            for (int k = 0; i + j + k < D; ++k) {
                ld v = a.c[i][j][k];
                if (v == 0) continue;
                r = add(r, scale(mul(mul(Xp[i], Yp[j]), Zp[k]), v));
            }
    return r;
}

// s^n P_n^{(alpha,0)}(t/s) as a polynomial, for polynomial t, s (three-term recurrence
// of the Jacobi polynomials with beta = 0, multiplied through by s^n).
std::vector<Poly> homog_jacobi(int nmax, int alpha, const Poly& t, const Poly& s) {
    std::vector<Poly> H(nmax + 1);
    H[0] = Poly::cst(1);
    if (nmax >= 1) H[1] = scale(add(scale(t, alpha + 2), scale(s, alpha)), 0.5L);
    Poly s2 = mul(s, s);
    for (int n = 2; n <= nmax; ++n) {
        ld a1 = 2.0L * n * (n + alpha) * (2 * n + alpha - 2);
        ld b = 2 * n + alpha - 1;
        ld c1 = (ld)(2 * n + alpha) * (2 * n + alpha - 2);
        ld a3 = 2.0L * (n + alpha - 1) * (n - 1) * (2 * n + alpha);
        Poly lin = add(scale(t, b * c1), scale(s, b * (ld)alpha * alpha));
        H[n] = scale(add(mul(lin, H[n - 1]), mul(s2, H[n - 2]), -a3), 1.0L / a1);
    }
    return H;
}

// Orthonormal Dubiner basis of P_p on the unit simplex of dimension d (d = 1, 2, 3),
// variables x, y, z, ordered by total degree (ties in (i, j, k) loop order); `deg`
// receives each function's degree.  psi_{ijk} has degree i + j + k and is orthogonal to
// every polynomial of lower degree, which makes the reference tables block-triangular
// in the degree (see build_ref_tables).
std::vector<Poly> dubiner(int d, int p, std::vector<int>* deg = nullptr) {
    Poly X = Poly::var(0), Y = Poly::var(1), Z = Poly::var(2), one = Poly::cst(1);
    std::vector<Poly> out;
    std::vector<int> dg;
    if (d == 1) {
        auto H = homog_jacobi(p, 0, add(scale(X, 2), one, -1), one);
        for (int i = 0; i <= p; ++i) {
            out.push_back(H[i]);
            dg.push_back(i);
        }
    } else if (d == 2) {
        Poly s1 = add(one, Y, -1), t1 = add(add(scale(X, 2), Y), one, -1);
        auto Hi = homog_jacobi(p, 0, t1, s1);
        for (int i = 0; i <= p; ++i) {
            auto Jj = homog_jacobi(p - i, 2 * i + 1, add(scale(Y, 2), one, -1), one);
            for (int j = 0; i + j <= p; ++j) {
                out.push_back(mul(Hi[i], Jj[j]));
                dg.push_back(i + j);
            }
        }
    } else {
        Poly s1 = add(add(one, Y, -1), Z, -1), t1 = add(add(add(scale(X, 2), Y), Z), one, -1);
        Poly s2 = add(one, Z, -1), t2 = add(add(scale(Y, 2), Z), one, -1);
        auto Hi = homog_jacobi(p, 0, t1, s1);
        for (int i = 0; i <= p; ++i) {
            auto Hj = homog_jacobi(p - i, 2 * i + 1, t2, s2);
            for (int j = 0; i + j <= p; ++j) {
                auto Jk = homog_jacobi(p - i - j, 2 * i + 2 * j + 2, add(scale(Z, 2), one, -1), one);
                Poly ij = mul(Hi[i], Hj[j]);
                for (int k = 0; i + j + k <= p; ++k) {
                    out.push_back(mul(ij, Jk[k]));
                    dg.push_back(i + j + k);
                }
            }
        }
    }
    for (auto& b : out) b = scale(b, 1.0L / std::sqrt(integrate(mul(b, b), d)));
    std::vector<int> order(out.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dg[a] < dg[b]; });
    std::vector<Poly> sorted;
    std::vector<int> sdeg;
    for (int i : order) {
        sorted.push_back(out[i]);
        sdeg.push_back(dg[i]);
    }
    if (deg) *deg = sdeg;
    return sorted;
}

Poly lambda_poly(int d, int j) {
    if (j == 0) {
        Poly r = Poly::cst(1);
        for (int l = 0; l < d; ++l) r = add(r, Poly::var(l), -1);
        return r;
    }
    return Poly::var(j - 1);
}

// affine parametrisation of facet f (opposite local vertex f) of the unit simplex by the
// unit (d-1)-simplex: x(s) = v_{i0} + sum_l s_l (v_{il} - v_{i0}), i0 < i1 < ... the other
// vertices; returns the d coordinate polynomials in the variables s = (x, y) slots.
void facet_map(int d, int f, Poly coord[3]) {
    int idx[3], n = 0;
    for (int i = 0; i <= d; ++i)
        if (i != f) idx[n++] = i;
    auto vert = [&](int i, int c) -> ld { return (i > 0 && c == i - 1) ? 1.0L : 0.0L; };
    for (int c = 0; c < 3; ++c) {
        if (c >= d) { coord[c] = Poly(); continue; }
        Poly r = Poly::cst(vert(idx[0], c));
        for (int l = 1; l < d; ++l) r = add(r, scale(Poly::var(l - 1), vert(idx[l], c) - vert(idx[0], c)));
        coord[c] = r;
    }
}

void invert(std::vector<ld>& A, int n) {
    std::vector<ld> I(n * n, 0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0) throw std::runtime_error("singular lattice Vandermonde");
        for (int k = 0; k < n; ++k) { std::swap(A[c * n + k], A[piv * n + k]); std::swap(I[c * n + k], I[piv * n + k]); }
        ld d = A[c * n + c];
        for (int k = 0; k < n; ++k) { A[c * n + k] /= d; I[c * n + k] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            ld f = A[r * n + c];
            if (f == 0) continue;
            for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
        }
    }
    A = I;
}

}  // namespace

RefTables build_ref_tables(int d, int p) {
    RefTables t;
    t.dim = d; t.p = p;
    std::vector<int> dpsi_deg, dchi_deg;
    auto psi = dubiner(d, p, &dpsi_deg);
    auto chi = dubiner(d - 1, p, &dchi_deg);
    const int nb = t.nb = (int)psi.size();
    const int nfb = t.nfb = (int)chi.size();
    std::vector<Poly> lam(d + 1), dpsi[3];
    for (int j = 0; j <= d; ++j) lam[j] = lambda_poly(d, j);
    for (int l = 0; l < d; ++l)
        for (int a = 0; a < nb; ++a) dpsi[l].push_back(deriv(psi[a], l));
    // orthonormality diagnostic
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) {
            double v = (double)integrate(mul(psi[a], psi[b]), d) - (a == b ? 1.0 : 0.0);
            t.max_orth_err = std::fmax(t.max_orth_err, std::fabs(v));
        }
    // volume: S[j][l][a][b] = int lambda_j psi_b d_l psi_a
    t.S.assign((size_t)(d + 1) * d * nb * nb, 0.0);
    for (int j = 0; j <= d; ++j)
        for (int b = 0; b < nb; ++b) {
            Poly lb = mul(lam[j], psi[b]);
            for (int l = 0; l < d; ++l)
                for (int a = 0; a < nb; ++a)
                    t.S[(((size_t)j * d + l) * nb + a) * nb + b] = (double)integrate(mul(lb, dpsi[l][a]), d);
        }
    // factored volume tables (c < nbm = dim P_{p-1}; the basis is ordered by degree)
    const int nbm = t.nbm = (int)std::count_if(dpsi_deg.begin(), dpsi_deg.end(), [&](int g) { return g < p; });
    t.D.assign((size_t)d * nbm * nb, 0.0);
    t.M.assign((size_t)(d + 1) * nbm * nb, 0.0);
    for (int l = 0; l < d; ++l)
        for (int c = 0; c < nbm; ++c)
            for (int a = 0; a < nb; ++a) t.D[((size_t)l * nbm + c) * nb + a] = (double)integrate(mul(psi[c], dpsi[l][a]), d);
    for (int j = 0; j <= d; ++j)
        for (int c = 0; c < nbm; ++c) {
            Poly lc = mul(lam[j], psi[c]);
            for (int b = 0; b < nb; ++b) t.M[((size_t)j * nbm + c) * nb + b] = (double)integrate(mul(lc, psi[b]), d);
        }
    // facets
    t.Tr.assign((size_t)(d + 1) * nfb * nb, 0.0);
    t.L.assign((size_t)(d + 1) * (d + 1) * nb * nfb, 0.0);
    for (int f = 0; f <= d; ++f) {
        Poly cm[3];
        facet_map(d, f, cm);
        std::vector<Poly> tr(nb), lamf(d + 1);
        for (int a = 0; a < nb; ++a) tr[a] = compose(psi[a], cm[0], cm[1], cm[2]);
        for (int j = 0; j <= d; ++j) lamf[j] = compose(lam[j], cm[0], cm[1], cm[2]);
        for (int c = 0; c < nfb; ++c)
            for (int a = 0; a < nb; ++a)
                t.Tr[((size_t)f * nfb + c) * nb + a] = (double)integrate(mul(chi[c], tr[a]), d - 1);
        for (int j = 0; j <= d; ++j) {
            if (j == f) continue;
            for (int a = 0; a < nb; ++a) {
                Poly la = mul(lamf[j], tr[a]);
                for (int c = 0; c < nfb; ++c)
                    t.L[(((size_t)j * (d + 1) + f) * nb + a) * nfb + c] = (double)integrate(mul(la, chi[c]), d - 1);
            }
        }
    }
    // Exact zeros left as rounding residue by the polynomial arithmetic: chi_c and psi_b are
    // orthogonal to every polynomial of lower degree, so S[j][l][a][b] = 0 for
    // deg b > deg a (lambda_j d_l psi_a has degree <= deg a), Tr[f][c][b] = 0 for
    // deg b < deg c, and L[j][f][a][c] = 0 for deg c > deg a + 1.  The tent kernels skip
    // these blocks; every table states them exactly.  Each entry set to zero must already be
    // rounding residue (checked: a wrong basis order must not silently change the operator).
    auto zero = [](double& v, double scale) {
        if (!(std::fabs(v) <= 1e-10 * scale)) throw std::runtime_error("reference tables: degree structure violated");
        v = 0.0;
    };
    // the tent kernels' loop bounds assume both bases in ascending degree
    if (!std::is_sorted(dpsi_deg.begin(), dpsi_deg.end()) || !std::is_sorted(dchi_deg.begin(), dchi_deg.end()))
        throw std::runtime_error("reference tables: basis not ordered by degree");
    double smax = 0, tmax = 0, lmax = 0;
    for (double v : t.S) smax = std::fmax(smax, std::fabs(v));
    for (double v : t.Tr) tmax = std::fmax(tmax, std::fabs(v));
    for (double v : t.L) lmax = std::fmax(lmax, std::fabs(v));
    for (int j = 0; j <= d; ++j)
        for (int l = 0; l < d; ++l)
            for (int a = 0; a < nb; ++a)
                for (int b = 0; b < nb; ++b)
                    if (dpsi_deg[b] > dpsi_deg[a]) zero(t.S[(((size_t)j * d + l) * nb + a) * nb + b], smax);
    for (int f = 0; f <= d; ++f)
        for (int c = 0; c < nfb; ++c)
            for (int b = 0; b < nb; ++b)
                if (dpsi_deg[b] < dchi_deg[c]) zero(t.Tr[((size_t)f * nfb + c) * nb + b], tmax);
    for (size_t jf = 0; jf < (size_t)(d + 1) * (d + 1); ++jf)
        for (int a = 0; a < nb; ++a)
            for (int c = 0; c < nfb; ++c)
                if (dchi_deg[c] > dpsi_deg[a] + 1) zero(t.L[(jf * nb + a) * nfb + c], lmax);
    // factored tables: D[l][c][a] = 0 unless deg c < deg a (d_l psi_a has degree deg a - 1);
    // M[j][c][b] = 0 unless |deg b - deg c| <= 1 (lambda_j psi_c has degree deg c + 1)
    double dmax = 0, mmax = 0;
    for (double v : t.D) dmax = std::fmax(dmax, std::fabs(v));
    for (double v : t.M) mmax = std::fmax(mmax, std::fabs(v));
    for (int l = 0; l < d; ++l)
        for (int c = 0; c < nbm; ++c)
            for (int a = 0; a < nb; ++a)
                if (dpsi_deg[c] >= dpsi_deg[a]) zero(t.D[((size_t)l * nbm + c) * nb + a], dmax);
    for (int j = 0; j <= d; ++j)
        for (int c = 0; c < nbm; ++c)
            for (int b = 0; b < nb; ++b)
                if (std::abs(dpsi_deg[b] - dpsi_deg[c]) > 1) zero(t.M[((size_t)j * nbm + c) * nb + b], mmax);
    // the factorisation reproduces S (an independent product of exact integrals)
    for (int j = 0; j <= d; ++j)
        for (int l = 0; l < d; ++l)
            for (int a = 0; a < nb; ++a)
                for (int b = 0; b < nb; ++b) {
                    ld acc = 0;
                    for (int c = 0; c < nbm; ++c)
                        acc += (ld)t.D[((size_t)l * nbm + c) * nb + a] * (ld)t.M[((size_t)j * nbm + c) * nb + b];
                    if (!(std::fabs((double)acc - t.S[(((size_t)j * d + l) * nb + a) * nb + b]) <= 1e-12 * smax))
                        throw std::runtime_error("reference tables: factored volume tables do not reproduce S");
                }
    // lattice Vandermonde (point order: i_d outermost, i_1 innermost)
    std::vector<ld> V((size_t)nb * nb);
    int k = 0;
    if (d == 2) {
        for (int i2 = 0; i2 <= p; ++i2)
            for (int i1 = 0; i1 + i2 <= p; ++i1, ++k)
                for (int a = 0; a < nb; ++a) V[(size_t)k * nb + a] = eval(psi[a], (ld)i1 / p, (ld)i2 / p, 0);
    } else {
        for (int i3 = 0; i3 <= p; ++i3)
            for (int i2 = 0; i2 + i3 <= p; ++i2)
                for (int i1 = 0; i1 + i2 + i3 <= p; ++i1, ++k)
                    for (int a = 0; a < nb; ++a)
                        V[(size_t)k * nb + a] = eval(psi[a], (ld)i1 / p, (ld)i2 / p, (ld)i3 / p);
    }
    t.V.assign(V.begin(), V.end());
    invert(V, nb);
    t.Vinv.assign(V.begin(), V.end());
    return t;
}

}  // namespace mtp
