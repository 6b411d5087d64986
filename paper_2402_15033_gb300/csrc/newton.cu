// Shifts of the Newton basis for the matrix powers kernel (host code).
//
// The paper runs its s-step GMRES with the monomial basis and names the Newton
// basis as the way to keep a large step size s well conditioned.  The Newton
// basis replaces A^i v by prod_i (A - theta_i I) v; good shifts are Ritz
// values of A in Leja order (Bai, Hu and Reichel, IMA J. Numer. Anal. 14,
// 1994): the solver's first restart cycle is standard GMRES (s = 1), whose
// k x k upper Hessenberg matrix H_k (A Q_k = Q_{k+1} H) has the Ritz values as
// eigenvalues.  Work here is O(k^3) on a k <= 63 matrix once per solve, so it
// runs on the host inside the library.
//
// * Eigenvalues: Francis double-shift QR on the Hessenberg matrix (Golub and
//   Van Loan, "Matrix Computations", the implicit double-shift QR step), with
//   deflation at negligible subdiagonals and an ad hoc exceptional shift after
//   10 and 20 unsuccessful sweeps.  Only the active diagonal window is
//   transformed: the eigenvalues do not depend on the rest.
// * Shifts: the real parts (a conjugate pair gives one real shift twice) in
//   Leja order, the first s, repeated cyclically when k < s.  The Leja order
//   scans the candidates in ascending order, starts at the largest modulus and
//   then takes the largest product of distances to the points already taken,
//   ties going to the first maximum; the distances are scaled by 2^-e with
//   max|z| <= 2^e so that the products neither overflow nor depend on the scale.
// * Scale: the power of two nearest (in log2) to the capacity of the interval
//   the shifts span, a quarter of its length, so that the shifted products
//   keep comparable norms.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>
#include "common.cuh"

namespace gm {
namespace {

// Householder reflector P = I - beta v v^T with v[0] = u[0] - alpha, P u = alpha e_1.
struct Reflector {
    double v[3];
    double beta;
    int len;
};

Reflector make_reflector(const double* u, int len) {
    Reflector r{};
    r.len = len;
    double nrm2 = 0.0;
    for (int i = 0; i < len; ++i) nrm2 += u[i] * u[i];
    double tail = 0.0;
    for (int i = 1; i < len; ++i) tail += u[i] * u[i];
    if (tail == 0.0 || !(nrm2 > 0.0)) {   // already a multiple of e_1: identity
        r.beta = 0.0;
        return r;
    }
    const double nrm = std::sqrt(nrm2);
    const double alpha = u[0] >= 0.0 ? -nrm : nrm;
    r.v[0] = u[0] - alpha;
    for (int i = 1; i < len; ++i) r.v[i] = u[i];
    double vv = 0.0;
    for (int i = 0; i < len; ++i) vv += r.v[i] * r.v[i];
    r.beta = 2.0 / vv;
    return r;
}

class Hess {
public:
    Hess(const double* H, int ldh, int k) : k_(k), a_((size_t)k * k) {
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < k; ++i) a_[i + (size_t)j * k] = (i <= j + 1) ? H[i + (size_t)j * ldh] : 0.0;
    }
    double& at(int i, int j) { return a_[i + (size_t)j * k_]; }

    // rows r0..r0+len-1, columns c0..c1: left multiply by P
    void left(const Reflector& p, int r0, int c0, int c1) {
        if (p.beta == 0.0) return;
        for (int j = c0; j <= c1; ++j) {
            double d = 0.0;
            for (int i = 0; i < p.len; ++i) d += p.v[i] * at(r0 + i, j);
            d *= p.beta;
            for (int i = 0; i < p.len; ++i) at(r0 + i, j) -= d * p.v[i];
        }
    }
    // columns c0..c0+len-1, rows r0..r1: right multiply by P
    void right(const Reflector& p, int c0, int r0, int r1) {
        if (p.beta == 0.0) return;
        for (int i = r0; i <= r1; ++i) {
            double d = 0.0;
            for (int j = 0; j < p.len; ++j) d += at(i, c0 + j) * p.v[j];
            d *= p.beta;
            for (int j = 0; j < p.len; ++j) at(i, c0 + j) -= d * p.v[j];
        }
    }

    // One implicit double-shift sweep over the window [l, h] (h - l >= 2),
    // shifts given by their sum and product.
    void francis_sweep(int l, int h, double ssum, double sprod) {
        double u[3];
        u[0] = at(l, l) * at(l, l) + at(l, l + 1) * at(l + 1, l) - ssum * at(l, l) + sprod;
        u[1] = at(l + 1, l) * (at(l, l) + at(l + 1, l + 1) - ssum);
        u[2] = at(l + 1, l) * at(l + 2, l + 1);
        for (int q = l; q <= h - 2; ++q) {
            const Reflector p = make_reflector(u, 3);
            left(p, q, std::max(l, q - 1), h);
            right(p, q, l, std::min(q + 3, h));
            if (q > l) {   // the bulge column is now alpha e_1 exactly
                at(q + 1, q - 1) = 0.0;
                at(q + 2, q - 1) = 0.0;
            }
            u[0] = at(q + 1, q);
            u[1] = at(q + 2, q);
            u[2] = (q < h - 2) ? at(q + 3, q) : 0.0;
        }
        const Reflector p = make_reflector(u, 2);
        left(p, h - 1, std::max(l, h - 2), h);
        right(p, h - 1, l, h);
        if (h - 2 >= l) at(h, h - 2) = 0.0;
    }

    // All k eigenvalues (re, im); false when an eigenvalue needs more than
    // kMaxSweeps sweeps.
    bool eigenvalues(std::vector<double>& re, std::vector<double>& im) {
        constexpr int kMaxSweeps = 60;
        const double eps = std::numeric_limits<double>::epsilon();
        re.assign(k_, 0.0);
        im.assign(k_, 0.0);
        double anorm = 0.0;
        for (double v : a_) anorm = std::max(anorm, std::fabs(v));
        for (double v : a_)
            if (!std::isfinite(v)) return false;
        // work on 2^-e H with anorm = f 2^e (exact): the sweep's squares and
        // products neither overflow nor underflow; the eigenvalues scale back
        int e = 0;
        if (anorm > 0.0) std::frexp(anorm, &e);
        for (double& v : a_) v = std::ldexp(v, -e);
        anorm = std::ldexp(anorm, -e);
        int h = k_ - 1, its = 0;
        while (h >= 0) {
            int l = h;
            for (; l > 0; --l) {
                double sc = std::fabs(at(l - 1, l - 1)) + std::fabs(at(l, l));
                if (sc == 0.0) sc = anorm;
                if (std::fabs(at(l, l - 1)) <= eps * sc) {
                    at(l, l - 1) = 0.0;
                    break;
                }
            }
            if (l == h) {
                re[h] = at(h, h);
                --h;
                its = 0;
                continue;
            }
            if (l == h - 1) {
                eig2(at(h - 1, h - 1), at(h - 1, h), at(h, h - 1), at(h, h), &re[h - 1], &im[h - 1], &re[h], &im[h]);
                h -= 2;
                its = 0;
                continue;
            }
            if (++its > kMaxSweeps) return false;
            double ssum, sprod;
            if (its == 10 || its == 20) {
                const double w = std::fabs(at(h, h - 1)) + std::fabs(at(h - 1, h - 2));
                ssum = 1.5 * w;
                sprod = w * w;
            } else {
                ssum = at(h - 1, h - 1) + at(h, h);
                sprod = at(h - 1, h - 1) * at(h, h) - at(h - 1, h) * at(h, h - 1);
            }
            francis_sweep(l, h, ssum, sprod);
        }
        for (int i = 0; i < k_; ++i) {
            re[i] = std::ldexp(re[i], e);
            im[i] = std::ldexp(im[i], e);
        }
        return true;
    }

private:
    // eigenvalues of [[a, b], [c, d]]: mid +- sqrt(p^2 + b c), p = (a - d) / 2,
    // the pair with the smaller magnitude root taken from the product
    static void eig2(double a, double b, double c, double d, double* r1, double* i1, double* r2, double* i2) {
        const double p = 0.5 * (a - d);
        const double disc = p * p + b * c;
        if (disc >= 0.0) {
            const double z = p + std::copysign(std::sqrt(disc), p);
            *r1 = d + z;
            *r2 = (z != 0.0) ? d - (b / z) * c : d;
            *i1 = *i2 = 0.0;
        } else {
            const double mid = d + p;
            const double w = std::sqrt(-disc);
            *r1 = *r2 = mid;
            *i1 = w;
            *i2 = -w;
        }
    }

    int k_;
    std::vector<double> a_;
};

}  // namespace

std::vector<double> leja_order(std::vector<double> x) {
    std::sort(x.begin(), x.end());
    const size_t n = x.size();
    std::vector<double> out;
    if (n == 0) return out;
    double top = 0.0;
    size_t first = 0;
    for (size_t i = 0; i < n; ++i)
        if (std::fabs(x[i]) > top) { top = std::fabs(x[i]); first = i; }
    int e = 0;
    if (top > 0.0) std::frexp(top, &e);
    const double scale = top > 0.0 ? std::ldexp(1.0, -e) : 1.0;
    std::vector<double> prod(n, 1.0);
    std::vector<char> left(n, 1);
    size_t last = first;
    left[last] = 0;
    out.push_back(x[last]);
    for (size_t t = 1; t < n; ++t) {
        double best = -1.0;
        size_t arg = 0;
        for (size_t i = 0; i < n; ++i) {
            prod[i] = prod[i] * std::fabs((x[i] - x[last]) * scale);
            const double cand = left[i] ? prod[i] : -1.0;
            if (cand > best) { best = cand; arg = i; }
        }
        last = arg;
        left[last] = 0;
        out.push_back(x[last]);
    }
    return out;
}

double newton_sigma(const double* theta, int s, double fallback) {
    if (s <= 0) return fallback;
    double lo = theta[0], hi = theta[0];
    for (int i = 1; i < s; ++i) { lo = std::min(lo, theta[i]); hi = std::max(hi, theta[i]); }
    const double cap = 0.25 * (hi - lo);
    if (!(cap > 0.0) || !std::isfinite(cap)) return fallback;
    int e = 0;
    const double f = std::frexp(cap, &e);
    return std::ldexp(1.0, f >= std::sqrt(0.5) ? e : e - 1);
}

int newton_shifts(const double* H, int ldh, int k, int s, double* theta) {
    if (k == 0) {
        for (int i = 0; i < s; ++i) theta[i] = 0.0;
        return GMRES_OK;
    }
    Hess hm(H, ldh, k);
    std::vector<double> re, im;
    if (!hm.eigenvalues(re, im)) {
        set_error("the QR iteration for the Ritz values did not converge (k = %d)", k);
        return GMRES_ERR_EIG;
    }
    const std::vector<double> pts = leja_order(re);
    for (int i = 0; i < s; ++i) theta[i] = pts[i % k];
    return GMRES_OK;
}

int chebyshev_interval(const double* H, int ldh, int k, double* c, double* delta) {
    *c = 0.0;
    *delta = 1.0;
    if (k == 0) return GMRES_OK;
    Hess hm(H, ldh, k);
    std::vector<double> re, im;
    if (!hm.eigenvalues(re, im)) {
        set_error("the QR iteration for the Ritz values did not converge (k = %d)", k);
        return GMRES_ERR_EIG;
    }
    const double lo = *std::min_element(re.begin(), re.end()), hi = *std::max_element(re.begin(), re.end());
    *c = 0.5 * (lo + hi);
    *delta = 0.5 * (hi - lo);
    // Ritz values without spread: delta = |c| (or 1), so that the basis stays defined
    if (!(*delta > 0.0) || !std::isfinite(*delta)) *delta = *c != 0.0 ? std::fabs(*c) : 1.0;
    return GMRES_OK;
}

}  // namespace gm

extern "C" {

int gmres_newton_shifts(const double* H, int32_t ldh, int32_t k, int32_t s, double* theta, double* sigma) {
    gm::clear_error();
    GM_ARG(k >= 0 && k <= 256, "k must be in [0, 256]");
    GM_ARG(s >= 1 && s <= 16, "s must be in [1, 16]");
    GM_ARG(k == 0 || (H != nullptr && ldh >= k), "H must be non-NULL with ldh >= k");
    GM_ARG(theta != nullptr, "theta is NULL");
    const int rc = gm::newton_shifts(H, ldh, k, s, theta);
    if (rc) return rc;
    if (sigma) *sigma = gm::newton_sigma(theta, s, *sigma);
    return GMRES_OK;
}

}  // extern "C"
