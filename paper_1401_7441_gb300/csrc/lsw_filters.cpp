// Filter tables of the least-asymmetric order-16 Daubechies basis (Sec. II.B), derived
// at context creation in double-double arithmetic and rounded once to FP64.
//
// Readings (the paper prints no coefficients):
//  * h: spectral factor of P(y) = sum_{k<8} C(7+k,k) y^k (|H(w)|^2 = 2 cos^16(w/2)
//    P(sin^2(w/2))); "least asymmetric" = smallest maximal deviation of the unwrapped
//    phase of the non-binomial factor Q(e^{-iw}) from its chord on [0, pi]; mirror
//    ties broken by first moment M_1 <= 1/2.  Support j = -7..8, sum h = sqrt 2.
//  * g_j = (-1)^j h_{1-j}.
//  * M_p = int x^p phi from the refinement equation.
//  * magic filter w_l (l = -7..8): sum_l w_l l^p = M_p, p = 0..15.
//  * kinetic: r_l = int phi phi''(. - l), r_l = 4 sum_n a_n r_{2l+n} (a = autocorrelation
//    of h), sum l^2 r_l = 2; blocks T_XY(l) = 4 sum X_k Y_k' r_{2l+k'-k}.
//  * forward filters (w*h)_m, (w*g)_m: synthesis to h/2 followed by the magic filter,
//    u_j = sum_i (w*h)_{j-2i} s_i + (w*g)_{j-2i} d_i.
//  * moment overlaps F^p(l) = int x^p phi phi(. - l), p <= 4, for the quartic confinement.
//
// Method: complex roots of P by the Durand-Kerner iteration in double, candidate
// filters in double, selection by the phase criterion, then Newton's method in
// double-double on the 16 defining equations (orthonormality of even shifts, eight
// vanishing moments of g) to full double-double accuracy.  Linear systems are solved
// by Gaussian elimination with partial pivoting in double-double.
//
// Double-double arithmetic: Dekker (1971) / Knuth error-free transformations (two-sum,
// fused-multiply two-product), normalised pairs (hi, lo) with |lo| <= ulp(hi)/2.
// This file must be compiled without floating-point contraction.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "lsw_internal.h"

namespace lsw {
namespace {

struct dd {
    double hi, lo;
};

inline dd mk(double a) { return {a, 0.0}; }
inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
inline dd fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}
inline dd two_prod(double a, double b) {
    double p = a * b;
    double e = std::fma(a, b, -p);
    return {p, e};
}
inline dd add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
inline dd neg(dd a) { return {-a.hi, -a.lo}; }
inline dd sub(dd a, dd b) { return add(a, neg(b)); }
inline dd mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
inline dd mul_d(dd a, double b) { return mul(a, mk(b)); }
inline dd div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = sub(a, mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = sub(r, mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return add(q, mk(q3));
}
inline dd dd_sqrt(dd a) {
    // one Newton step on y = sqrt(a) from the FP64 estimate
    double y = std::sqrt(a.hi);
    dd y2 = two_prod(y, y);
    dd r = sub(a, y2);
    return add(mk(y), mk(r.hi / (2.0 * y)));
}
inline double to_d(dd a) { return a.hi + a.lo; }
inline double absd(dd a) { return std::fabs(a.hi); }

// Gaussian elimination with partial pivoting, A (n x n row-major) x = b, in dd.
bool solve(std::vector<dd> A, std::vector<dd> b, int n, std::vector<dd>* x) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (absd(A[r * n + c]) > absd(A[p * n + c])) p = r;
        if (absd(A[p * n + c]) == 0.0) return false;
        if (p != c) {
            for (int k = 0; k < n; ++k) std::swap(A[p * n + k], A[c * n + k]);
            std::swap(b[p], b[c]);
        }
        for (int r = c + 1; r < n; ++r) {
            dd f = div(A[r * n + c], A[c * n + c]);
            if (f.hi == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] = sub(A[r * n + k], mul(f, A[c * n + k]));
            b[r] = sub(b[r], mul(f, b[c]));
        }
    }
    x->assign(n, mk(0.0));
    for (int r = n - 1; r >= 0; --r) {
        dd s = b[r];
        for (int k = r + 1; k < n; ++k) s = sub(s, mul(A[r * n + k], (*x)[k]));
        (*x)[r] = div(s, A[r * n + r]);
    }
    return true;
}

using cplx = std::complex<double>;

// Durand-Kerner iteration for the roots of a monic polynomial sum_k c[k] y^k.
std::vector<cplx> poly_roots(const std::vector<double>& c) {
    const int n = static_cast<int>(c.size()) - 1;
    std::vector<cplx> z(n);
    const cplx seed(0.4, 0.9);
    for (int i = 0; i < n; ++i) z[i] = std::pow(seed, i);
    auto eval = [&](cplx y) {
        cplx v = c[n];
        for (int k = n - 1; k >= 0; --k) v = v * y + c[k];
        return v;
    };
    for (int it = 0; it < 2000; ++it) {
        double moved = 0.0;
        for (int i = 0; i < n; ++i) {
            cplx den = 1.0;
            for (int j = 0; j < n; ++j)
                if (j != i) den *= (z[i] - z[j]);
            cplx dz = eval(z[i]) / den;
            z[i] -= dz;
            moved = std::max(moved, std::abs(dz));
        }
        if (moved < 1e-16) break;
    }
    // Newton polish on the original polynomial
    for (int i = 0; i < n; ++i) {
        for (int it = 0; it < 4; ++it) {
            cplx v = c[n], dv = 0.0;
            for (int k = n - 1; k >= 0; --k) {
                dv = dv * z[i] + v;
                v = v * z[i] + c[k];
            }
            if (std::abs(dv) > 0) z[i] -= v / dv;
        }
    }
    return z;
}

// Maximal deviation of the unwrapped phase of Q(e^{-iw}) from its chord on [0, pi].
double phase_deviation(const std::vector<double>& q) {
    const int S = 1024;
    const double pi = 3.14159265358979323846;
    std::vector<double> th(S + 1);
    double prev = 0.0;
    for (int k = 0; k <= S; ++k) {
        double w = pi * k / S;
        cplx v = 0.0;
        for (size_t i = 0; i < q.size(); ++i) v += q[i] * std::exp(cplx(0.0, -w * static_cast<double>(i)));
        double a = std::arg(v);
        while (a - prev > pi) a -= 2 * pi;
        while (a - prev < -pi) a += 2 * pi;
        th[k] = a;
        prev = a;
    }
    double dev = 0.0;
    for (int k = 0; k <= S; ++k) dev = std::max(dev, std::fabs(th[k] - th[S] * k / S));
    return dev;
}

std::vector<cplx> polymul(const std::vector<cplx>& a, const std::vector<cplx>& b) {
    std::vector<cplx> r(a.size() + b.size() - 1, 0.0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
    return r;
}

double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

bool least_asymmetric(std::vector<double>* h_out, std::string* err) {
    const int m = 8;
    std::vector<double> c(m);
    for (int k = 0; k < m; ++k) c[k] = binom(m - 1 + k, k);
    const double lead = c[m - 1];
    for (auto& v : c) v /= lead;
    std::vector<cplx> y = poly_roots(c);
    // groups: real roots and the Im > 0 member of each conjugate pair
    std::vector<std::pair<bool, cplx>> groups;
    for (auto& r : y) {
        if (std::fabs(r.imag()) < 1e-9)
            groups.push_back({true, cplx(r.real(), 0.0)});
        else if (r.imag() > 0)
            groups.push_back({false, r});
    }
    if (groups.size() != 4) {
        *err = "unexpected root structure of the Daubechies polynomial";
        return false;
    }
    struct Cand {
        double dev, m1;
        std::vector<double> h;
    };
    std::vector<Cand> cands;
    for (int bits = 0; bits < (1 << groups.size()); ++bits) {
        std::vector<cplx> q{1.0};
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            cplx yy = groups[gi].second;
            cplx b = 2.0 - 4.0 * yy;
            cplx d = std::sqrt(b * b - 4.0);
            cplx z1 = (b + d) / 2.0, z2 = (b - d) / 2.0;
            cplx in = std::abs(z1) < std::abs(z2) ? z1 : z2;
            cplx out = std::abs(z1) < std::abs(z2) ? z2 : z1;
            cplx z = ((bits >> gi) & 1) ? out : in;
            if (groups[gi].first) {
                q = polymul(q, {-cplx(z.real(), 0.0), 1.0});
            } else {
                q = polymul(q, {-z, 1.0});
                q = polymul(q, {-std::conj(z), 1.0});
            }
        }
        std::vector<double> qr(q.size());
        double sq = 0.0;
        for (size_t i = 0; i < q.size(); ++i) {
            qr[i] = q[i].real();
            sq += qr[i];
        }
        if (sq < 0)
            for (auto& v : qr) v = -v;
        std::vector<cplx> full(qr.begin(), qr.end());
        for (int k = 0; k < m; ++k) full = polymul(full, {1.0, 1.0});
        double s = 0.0;
        for (auto& v : full) s += v.real();
        Cand cd;
        cd.h.resize(full.size());
        for (size_t i = 0; i < full.size(); ++i) cd.h[i] = full[i].real() * std::sqrt(2.0) / s;
        double m1 = 0.0;
        for (int i = 0; i < D16; ++i) m1 += (i + H_LO) * cd.h[i];
        cd.m1 = m1 * std::sqrt(2.0) / 2.0;
        cd.dev = phase_deviation(qr);
        cands.push_back(cd);
    }
    double best = 1e300;
    for (auto& cd : cands) best = std::min(best, cd.dev);
    const Cand* pick = nullptr;
    int ties = 0;
    for (auto& cd : cands) {
        if (cd.dev <= best * (1 + 1e-9) && cd.m1 <= 0.5) {
            pick = &cd;
            ++ties;
        }
    }
    if (!pick || ties != 1) {
        *err = "least-asymmetric factor not unique";
        return false;
    }
    *h_out = pick->h;
    return true;
}

// Newton's method in dd on F(h) = 0: sum_j h_j h_{j+2k} - delta_k (k = 0..7),
// sum_j (-1)^j j^p h_j (p = 0..7); moment rows scaled to unit max coefficient.
bool polish(const std::vector<double>& h0, std::vector<dd>* hout, std::string* err) {
    const int n = D16;
    std::vector<dd> h(n);
    for (int i = 0; i < n; ++i) h[i] = mk(h0[i]);
    std::vector<double> mrow(8 * n);
    for (int p = 0; p < 8; ++p) {
        double mx = 0.0;
        for (int i = 0; i < n; ++i) {
            int j = i + H_LO;
            double v = ((j % 2 == 0) ? 1.0 : -1.0) * std::pow(static_cast<double>(j), p);
            mrow[p * n + i] = v;
            mx = std::max(mx, std::fabs(v));
        }
        for (int i = 0; i < n; ++i) mrow[p * n + i] /= mx;  // exact scaling not required
    }
    for (int it = 0; it < 8; ++it) {
        std::vector<dd> F(n), Jm(n * n, mk(0.0));
        for (int k = 0; k < 8; ++k) {
            dd s = mk(k == 0 ? -1.0 : 0.0);
            for (int i = 0; i + 2 * k < n; ++i) s = add(s, mul(h[i], h[i + 2 * k]));
            F[k] = s;
            for (int i = 0; i < n; ++i) {
                dd v = mk(0.0);
                if (i + 2 * k < n) v = add(v, h[i + 2 * k]);
                if (i - 2 * k >= 0) v = add(v, h[i - 2 * k]);
                Jm[k * n + i] = v;
            }
        }
        for (int p = 0; p < 8; ++p) {
            dd s = mk(0.0);
            for (int i = 0; i < n; ++i) s = add(s, mul_d(h[i], mrow[p * n + i]));
            F[8 + p] = s;
            for (int i = 0; i < n; ++i) Jm[(8 + p) * n + i] = mk(mrow[p * n + i]);
        }
        std::vector<dd> dx;
        if (!solve(Jm, F, n, &dx)) {
            *err = "singular Newton system for the Daubechies filter";
            return false;
        }
        for (int i = 0; i < n; ++i) h[i] = sub(h[i], dx[i]);
    }
    *hout = h;
    return true;
}

}  // namespace

bool derive_filters(FilterSet* out, std::string* err) {
    std::vector<double> h0;
    if (!least_asymmetric(&h0, err)) return false;
    std::vector<dd> h;
    if (!polish(h0, &h, err)) return false;
    const int n = D16;
    std::vector<dd> g(n);
    for (int i = 0; i < n; ++i) {
        int j = i + H_LO;
        int src = (1 - j) - H_LO;  // h_{1-j}
        g[i] = (j % 2 == 0) ? h[src] : neg(h[src]);
    }
    const dd sqrt2 = dd_sqrt(mk(2.0));

    // moments: M_p (1 - 2^-p) = 2^(-p-1) sqrt2 sum_{i<p} C(p,i) M_i sum_j h_j j^(p-i)
    std::vector<dd> hm(n);
    for (int q = 0; q < n; ++q) {
        dd s = mk(0.0);
        for (int i = 0; i < n; ++i) {
            dd jp = mk(1.0);
            for (int r = 0; r < q; ++r) jp = mul_d(jp, static_cast<double>(i + H_LO));
            s = add(s, mul(h[i], jp));
        }
        hm[q] = s;
    }
    std::vector<dd> M(n);
    M[0] = mk(1.0);
    for (int p = 1; p < n; ++p) {
        dd acc = mk(0.0);
        for (int i = 0; i < p; ++i) acc = add(acc, mul(mul_d(M[i], binom(p, i)), hm[p - i]));
        dd den = mk(std::ldexp(1.0, p + 1) * (1.0 - std::ldexp(1.0, -p)));
        M[p] = div(mul(sqrt2, acc), den);
    }

    // magic filter, conditioned form: nodes t_l = (l - 1/2) / 7.5, moments about 1/2
    std::vector<dd> mu(n);
    for (int p = 0; p < n; ++p) {
        dd s = mk(0.0);
        for (int i = 0; i <= p; ++i) {
            dd term = mul_d(M[i], binom(p, i));
            for (int r = 0; r < p - i; ++r) term = mul_d(term, -0.5);
            s = add(s, term);
        }
        for (int r = 0; r < p; ++r) s = div(s, mk(7.5));
        mu[p] = s;
    }
    std::vector<dd> V(n * n);
    for (int p = 0; p < n; ++p)
        for (int l = 0; l < n; ++l) {
            dd t = div(mk((l + H_LO) - 0.5), mk(7.5));
            dd v = mk(1.0);
            for (int r = 0; r < p; ++r) v = mul(v, t);
            V[p * n + l] = v;
        }
    std::vector<dd> w;
    if (!solve(V, mu, n, &w)) {
        *err = "singular magic-filter system";
        return false;
    }

    // connection coefficients with r_{-l} = r_l: unknowns r_0..r_14; equations
    // r_l - 4 sum_n a_n r_{|2l+n|} = 0 for l = 0..13, and 2 sum_{l>=1} l^2 r_l = 2
    const int L = KIN_HALF;
    std::vector<dd> ac(2 * n - 1, mk(0.0));  // a_d, d = -(n-1)..n-1
    for (int d = -(n - 1); d <= n - 1; ++d) {
        dd s = mk(0.0);
        for (int i = 0; i < n; ++i)
            if (i + d >= 0 && i + d < n) s = add(s, mul(h[i], h[i + d]));
        ac[d + n - 1] = s;
    }
    const int nu = L + 1;
    std::vector<dd> A(nu * nu, mk(0.0)), b(nu, mk(0.0));
    for (int l = 0; l < L; ++l) {
        A[l * nu + l] = add(A[l * nu + l], mk(1.0));
        for (int d = -(n - 1); d <= n - 1; ++d) {
            int m2 = std::abs(2 * l + d);
            if (m2 > L) continue;
            A[l * nu + m2] = sub(A[l * nu + m2], mul_d(ac[d + n - 1], 4.0));
        }
    }
    for (int l = 1; l <= L; ++l) A[L * nu + l] = mk(2.0 * l * l);
    b[L] = mk(2.0);
    std::vector<dd> rs;
    if (!solve(A, b, nu, &rs)) {
        *err = "singular connection-coefficient system";
        return false;
    }
    std::vector<dd> r(KIN_TAPS);
    for (int l = -L; l <= L; ++l) r[l + L] = rs[std::abs(l)];

    // kinetic blocks
    const std::vector<dd>* XY[2] = {&h, &g};
    dd T[4][KIN_TAPS];
    for (int bx = 0; bx < 2; ++bx)
        for (int by = 0; by < 2; ++by)
            for (int l = -L; l <= L; ++l) {
                dd s = mk(0.0);
                for (int k = 0; k < n; ++k)
                    for (int kp = 0; kp < n; ++kp) {
                        int m = 2 * l + (kp + H_LO) - (k + H_LO);
                        if (m < -L || m > L) continue;
                        s = add(s, mul(mul((*XY[bx])[k], (*XY[by])[kp]), r[m + L]));
                    }
                T[bx * 2 + by][l + L] = mul_d(s, 4.0);
            }

    // moment overlaps F^p(l) = int x^p phi(x) phi(x - l) dx, p = 0..4, |l| <= 14 (the 1D
    // Galerkin entries of the multiplication operators x^p, which the quartic confining
    // potential needs): the refinement equation in both factors and x = (y + k) / 2 give
    //   F^p(l) = 2^-p sum_{k,k'} h_k h_k' sum_{q<=p} C(p,q) k^(p-q) F^q(2l + k' - k);
    // F^0 = delta (orthonormal translates); for p >= 1 the q = p part moves to the left,
    // (I - 2^-p A) F^p = 2^-p sum_{q<p} ..., A(l, m) = a_{m - 2l} (autocorrelation of h).
    std::vector<std::vector<dd>> Fm(MOVL_P, std::vector<dd>(KIN_TAPS, mk(0.0)));
    Fm[0][L] = mk(1.0);
    for (int p = 1; p < MOVL_P; ++p) {
        std::vector<dd> Am(KIN_TAPS * KIN_TAPS, mk(0.0)), bm(KIN_TAPS, mk(0.0));
        const double sc = std::ldexp(1.0, -p);
        for (int l = -L; l <= L; ++l) {
            for (int m = -L; m <= L; ++m) {
                const int d = m - 2 * l;
                dd v = (d >= -(n - 1) && d <= n - 1) ? mul_d(ac[d + n - 1], -sc) : mk(0.0);
                if (m == l) v = add(v, mk(1.0));
                Am[(l + L) * KIN_TAPS + (m + L)] = v;
            }
            dd acc = mk(0.0);
            for (int q = 0; q < p; ++q)
                for (int k = 0; k < n; ++k)
                    for (int kp = 0; kp < n; ++kp) {
                        const int idx = 2 * l + (kp + H_LO) - (k + H_LO);
                        if (idx < -L || idx > L) continue;
                        dd t = mul(mul(h[k], h[kp]), Fm[q][idx + L]);
                        for (int r = 0; r < p - q; ++r) t = mul_d(t, static_cast<double>(k + H_LO));
                        acc = add(acc, mul_d(t, binom(p, q)));
                    }
            bm[l + L] = mul_d(acc, sc);
        }
        if (!solve(Am, bm, KIN_TAPS, &Fm[p])) {
            *err = "singular moment-overlap system";
            return false;
        }
    }

    // forward filters (w * X)_m, m = -14..16
    dd Fw[2][FWD_TAPS];
    for (int x = 0; x < 2; ++x)
        for (int m = FWD_LO; m < FWD_LO + FWD_TAPS; ++m) {
            dd s = mk(0.0);
            for (int k = 0; k < n; ++k) {
                int l = m - (k + H_LO);
                if (l < H_LO || l >= H_LO + n) continue;
                s = add(s, mul(w[l - H_LO], (*XY[x])[k]));
            }
            Fw[x][m - FWD_LO] = s;
        }

    for (int i = 0; i < n; ++i) {
        out->h[i] = to_d(h[i]);
        out->g[i] = to_d(g[i]);
        out->moments[i] = to_d(M[i]);
        out->magic[i] = to_d(w[i]);
    }
    for (int i = 0; i < KIN_TAPS; ++i) {
        out->kin_r[i] = to_d(r[i]);
        for (int k = 0; k < 4; ++k) out->kin[k][i] = to_d(T[k][i]);
    }
    for (int x = 0; x < 2; ++x)
        for (int i = 0; i < FWD_TAPS; ++i) out->fwd[x][i] = to_d(Fw[x][i]);
    for (int p = 0; p < MOVL_P; ++p)
        for (int i = 0; i < KIN_TAPS; ++i) out->movl[p][i] = to_d(Fm[p][i]);
    return true;
}

}  // namespace lsw
