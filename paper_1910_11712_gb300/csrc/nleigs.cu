// NLEIGS, static variant (Sec. 4.5): a rational interpolant R_d(z) = sum_j b_j(z) D_j of the
// split operator on a target set Sigma (the region's ellipse), linearised as the pencil (A, B)
// of Sec. 4.5.1 Eq. (nleigsmatlin) with d blocks of n, and shift-and-invert Arnoldi on
// S = (A - sigma B)^{-1} B with a full (d n)-vector basis.
//
// Host (small, FP64):
//   * the boundary of Sigma at nb points, the singularity set Xi from the function trees
//     (denominator roots of rational nodes and of a quotient's rational denominator, square-root
//     cuts sampled at fixed distances; exp has none);
//   * Leja-Bagby nodes sigma_j and poles xi_j (Sec. 4.5.1 Eq. (nleigsleja)), scalings beta_j
//     with max |b_j| = 1 on the boundary (Eq. (nleigsbj));
//   * scalar divided differences d_i^j = e_j^T f_i(H K^{-1}) e_1 (Eq. (nleigsfdd)) through
//     functions of the lower-triangular H K^{-1}: matrix polynomials and triangular solves,
//     exp by scaling and squaring of its Taylor series, sqrt by the Bjorck-Hammarling
//     recurrence (the interpolation recurrence of Eq. (nleigsdd) loses digits to cancellation
//     at about eps max|f| on the boundary, which decided the degree test); the degree: the first
//     d >= 1 whose last pole, taken as infinity, gives max_i |d_i^d| < tol max_i |d_i^0|.
// Device (FP64), one Arnoldi step w = S v (Sec. 4.5.2, Eqs. (nleigstoarreca), (nleigstoarrecb)):
//   * with z = B v (z^j = v^{j-1} + beta_j/xi_j v^j), a particular solution p of the block rows
//     1..d-1 with p^{d-1} = 0, p^{j-1} = (z^j - beta_j (1 - sigma/xi_j) p^j) / (sigma_{j-1} - sigma),
//     and the per-term combinations c_i = sum_{j<=d-2} d_i^j p^j + d_i^d / beta_d v^{d-1}, one
//     thread per row (nleigs_expand_kernel);
//   * u = R_d(sigma)^{-1} (-sum_i A_i c_i): the split SpMV, then the band LU of R_d(sigma)
//     (= sum_i (sum_j b_j(sigma) d_i^j) A_i, factored once in complex64) with the substitution
//     sweeps and two corrections against the FP64 residual of R_d(sigma);
//   * w^j = p^j + b_j(sigma) u (the null space of the lower block rows is b(sigma) (x) C^n);
//   * classical Gram-Schmidt, twice, against the basis (FP64 dot and update kernels).
// The Ritz pairs of the Hessenberg matrix give lambda = sigma + 1/theta with x the first block of
// the Ritz vector; the pairs inside Sigma are accepted by the FP64 scaled residual of the full
// T (not of R_d) like the contour method's.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "nep_common.cuh"

namespace nep {

namespace {

typedef std::complex<double> cd;

inline cd to_cd(zd z) { return cd(z.re, z.im); }
inline zd to_zd(cd z) { return mk(z.real(), z.imag()); }

// roots of c[0] x^m + ... + c[m] (c[0] the leading coefficient) by Durand-Kerner iteration
std::vector<cd> poly_roots(std::vector<cd> c) {
    while (!c.empty() && c.front() == cd(0.0)) c.erase(c.begin());
    const int m = (int)c.size() - 1;
    std::vector<cd> r;
    if (m < 1) return r;
    for (int k = 1; k <= m; ++k) c[k] /= c[0];
    c[0] = 1.0;
    if (m == 1) return {-c[1]};
    double rad = 0.0;
    for (int k = 1; k <= m; ++k) rad = std::max(rad, std::pow(std::abs(c[k]), 1.0 / k));
    rad = 1.0 + rad;
    for (int k = 0; k < m; ++k) r.push_back(rad * std::pow(cd(0.4, 0.9), k));
    auto p = [&](cd x) {
        cd v = 1.0;
        for (int k = 1; k <= m; ++k) v = v * x + c[k];
        return v;
    };
    for (int it = 0; it < 2000; ++it) {
        double move = 0.0;
        for (int k = 0; k < m; ++k) {
            cd den = 1.0;
            for (int j = 0; j < m; ++j)
                if (j != k) den *= r[k] - r[j];
            if (den == cd(0.0)) den = cd(1e-300);
            const cd step = p(r[k]) / den;
            r[k] -= step;
            move = std::max(move, std::abs(step) / std::max(1.0, std::abs(r[k])));
        }
        if (move < 1e-16) break;
    }
    return r;
}

std::vector<cd> coef_slice(const std::vector<zd>& pool, int off, int len) {
    std::vector<cd> c;
    for (int t = 0; t < len; ++t) c.push_back(to_cd(pool[off + t]));
    return c;
}

// singular points in z of node k whose input is scale * z
void node_singularities(const std::vector<FnNode>& nodes, const std::vector<zd>& pool, int k, cd scale,
                        const std::vector<double>& cut_t, std::vector<cd>* out, int depth) {
    if (k < 0 || k >= (int)nodes.size() || depth > 16) return;
    const FnNode& nd = nodes[k];
    const cd s = to_cd(nd.alpha) * scale;  // the node's inner argument is s z
    if (nd.kind == NEP_FN_RATIONAL) {
        if (nd.den_len > 1)
            for (cd r : poly_roots(coef_slice(pool, nd.den_off, nd.den_len))) out->push_back(r / s);
    } else if (nd.kind == NEP_FN_SQRT) {
        for (double t : cut_t) out->push_back((to_cd(nd.shift) - t) / s);
    } else if (nd.kind == NEP_FN_COMBINE) {
        if (nd.op == NEP_OP_COMPOSE) {
            node_singularities(nodes, pool, nd.b, s, cut_t, out, depth + 1);
        } else {
            node_singularities(nodes, pool, nd.a, s, cut_t, out, depth + 1);
            node_singularities(nodes, pool, nd.b, s, cut_t, out, depth + 1);
            if (nd.op == NEP_OP_DIV && nd.b >= 0 && nodes[nd.b].kind == NEP_FN_RATIONAL && nodes[nd.b].num_len > 1) {
                const cd sb = to_cd(nodes[nd.b].alpha) * s;
                for (cd r : poly_roots(coef_slice(pool, nodes[nd.b].num_off, nodes[nd.b].num_len)))
                    out->push_back(r / sb);
            }
        }
    }
}

const double kInf = INFINITY;
inline bool finite_pole(cd x) { return std::isfinite(x.real()) && std::isfinite(x.imag()); }

// b_0 .. b_d at z (b_0 = 1/beta_0)
void basis_at(cd z, const std::vector<cd>& sig, const std::vector<cd>& xi, const std::vector<double>& beta, int d,
              std::vector<cd>* b) {
    b->assign(d + 1, 0.0);
    (*b)[0] = 1.0 / beta[0];
    for (int j = 1; j <= d; ++j) {
        cd g = (*b)[j - 1] * (z - sig[j - 1]) / beta[j];
        if (finite_pole(xi[j])) g /= (1.0 - z / xi[j]);
        (*b)[j] = g;
    }
}

// ---- functions of small lower-triangular matrices (the divided differences of Sec. 4.5.1
// Eq. (nleigsfdd)): every matrix here is a function of one lower-triangular M, so all of them are
// lower triangular and commute
struct LMat {
    int m = 0;
    std::vector<cd> a;  // column-major, entries above the diagonal stay zero
    explicit LMat(int m_ = 0) : m(m_), a((size_t)m_ * m_, 0.0) {}
    cd& operator()(int i, int j) { return a[i + (size_t)m * j]; }
    cd operator()(int i, int j) const { return a[i + (size_t)m * j]; }
};

LMat lm_eye(int m, cd v = 1.0) {
    LMat r(m);
    for (int i = 0; i < m; ++i) r(i, i) = v;
    return r;
}
LMat lm_mul(const LMat& A, const LMat& B) {
    LMat C(A.m);
    for (int j = 0; j < A.m; ++j)
        for (int i = j; i < A.m; ++i) {
            cd acc = 0.0;
            for (int k = j; k <= i; ++k) acc += A(i, k) * B(k, j);
            C(i, j) = acc;
        }
    return C;
}
LMat lm_axpby(cd x, const LMat& A, cd y, const LMat& B) {
    LMat C(A.m);
    for (size_t t = 0; t < C.a.size(); ++t) C.a[t] = x * A.a[t] + y * B.a[t];
    return C;
}
// L^{-1} B for lower-triangular L (forward substitution, column by column)
LMat lm_solve(const LMat& L, const LMat& B) {
    LMat X(B.m);
    for (int j = 0; j < B.m; ++j)
        for (int i = j; i < B.m; ++i) {
            cd acc = B(i, j);
            for (int k = j; k < i; ++k) acc -= L(i, k) * X(k, j);
            X(i, j) = acc / L(i, i);
        }
    return X;
}
LMat lm_poly(const std::vector<cd>& c, const LMat& X) {  // c[0] the leading coefficient (Horner)
    LMat R(X.m);
    for (cd a : c) R = lm_axpby(1.0, lm_mul(R, X), 1.0, lm_eye(X.m, a));
    return R;
}
// exp by scaling and squaring of the Taylor series: ||X / 2^s||_1 <= 1/2, 20 terms (truncation
// below (1/2)^21 / 21!, far under the rounding of the squarings)
LMat lm_exp(const LMat& X) {
    double nrm = 0.0;
    for (int j = 0; j < X.m; ++j) {
        double cs = 0.0;
        for (int i = j; i < X.m; ++i) cs += std::abs(X(i, j));
        nrm = std::max(nrm, cs);
    }
    int sq = 0;
    while (nrm > 0.5 && sq < 60) {
        nrm *= 0.5;
        ++sq;
    }
    const LMat Y = lm_axpby(std::ldexp(1.0, -sq), X, 0.0, X);
    LMat E = lm_eye(X.m), term = lm_eye(X.m);
    for (int k = 1; k <= 20; ++k) {
        term = lm_axpby(1.0 / k, lm_mul(term, Y), 0.0, term);
        E = lm_axpby(1.0, E, 1.0, term);
    }
    for (int k = 0; k < sq; ++k) E = lm_mul(E, E);
    return E;
}
// principal square root of a lower-triangular T by the Bjorck-Hammarling recurrence, diagonal by
// diagonal: R_ii = sqrt(T_ii), R_ij = (T_ij - sum_{j<k<i} R_ik R_kj) / (R_ii + R_jj)
LMat lm_sqrt(const LMat& T) {
    LMat R(T.m);
    for (int i = 0; i < T.m; ++i) R(i, i) = std::sqrt(T(i, i));
    for (int dist = 1; dist < T.m; ++dist)
        for (int j = 0; j + dist < T.m; ++j) {
            const int i = j + dist;
            cd acc = T(i, j);
            for (int k = j + 1; k < i; ++k) acc -= R(i, k) * R(k, j);
            R(i, j) = acc / (R(i, i) + R(j, j));
        }
    return R;
}

// f_k(M) for the function tree at node k: beta h(alpha M)
LMat lm_fn(const std::vector<FnNode>& nodes, const std::vector<zd>& pool, int k, const LMat& M, int depth) {
    const FnNode& nd = nodes[k];
    const LMat X = lm_axpby(to_cd(nd.alpha), M, 0.0, M);
    LMat H(M.m);
    if (nd.kind == NEP_FN_RATIONAL) {
        H = lm_poly(coef_slice(pool, nd.num_off, nd.num_len), X);
        if (nd.den_len > 0) H = lm_solve(lm_poly(coef_slice(pool, nd.den_off, nd.den_len), X), H);
    } else if (nd.kind == NEP_FN_EXP) {
        H = lm_exp(X);
    } else if (nd.kind == NEP_FN_SQRT) {
        H = lm_sqrt(lm_axpby(1.0, X, -1.0, lm_eye(M.m, to_cd(nd.shift))));
    } else if (depth <= 16) {
        if (nd.op == NEP_OP_COMPOSE) {
            H = lm_fn(nodes, pool, nd.a, lm_fn(nodes, pool, nd.b, X, depth + 1), depth + 1);
        } else {
            const LMat A = lm_fn(nodes, pool, nd.a, X, depth + 1), B = lm_fn(nodes, pool, nd.b, X, depth + 1);
            if (nd.op == NEP_OP_ADD) H = lm_axpby(1.0, A, 1.0, B);
            else if (nd.op == NEP_OP_MUL) H = lm_mul(A, B);
            else H = lm_solve(B, A);  // A B^{-1} = B^{-1} A: they commute
        }
    }
    return lm_axpby(to_cd(nd.beta), H, 0.0, H);
}

}  // namespace

int nleigs_interpolation(const std::vector<FnNode>& nodes, const std::vector<zd>& pool, const std::vector<int>& roots,
                         zd c, double a, double b, double tol, int dmax, int nb, NleigsInterp* out) {
    const int nt = (int)roots.size();
    std::vector<cd> bnd(nb);
    for (int k = 0; k < nb; ++k) {
        const double th = 6.283185307179586476925 * k / nb;
        bnd[k] = to_cd(c) + cd(a * std::cos(th), b * std::sin(th));
    }
    std::vector<double> cut_t{0.0};
    for (int k = 0; k < 48; ++k) cut_t.push_back(std::pow(10.0, -4.0 + 8.0 * k / 47.0));
    std::vector<cd> Xi;
    for (int i = 0; i < nt; ++i) node_singularities(nodes, pool, roots[i], 1.0, cut_t, &Xi, 0);
    // Leja-Bagby: s_j on the boundary and on Xi, rescaled to max 1 on the boundary every step
    std::vector<cd> sig(dmax + 1), xin(dmax + 1, cd(kInf, 0.0));
    std::vector<char> used(Xi.size(), 0);
    sig[0] = bnd[0];
    std::vector<cd> sb(nb), sx(Xi.size());
    for (int k = 0; k < nb; ++k) sb[k] = bnd[k] - sig[0];
    for (size_t k = 0; k < Xi.size(); ++k) sx[k] = Xi[k] - sig[0];
    for (int j = 0; j < dmax; ++j) {
        int kb = 0;
        for (int k = 1; k < nb; ++k)
            if (std::abs(sb[k]) > std::abs(sb[kb])) kb = k;
        sig[j + 1] = bnd[kb];
        int kx = -1;
        for (size_t k = 0; k < Xi.size(); ++k) {
            const double v = std::abs(sx[k]);
            if (used[k] || !std::isfinite(v)) continue;
            if (kx < 0 || v < std::abs(sx[kx])) kx = (int)k;
        }
        if (kx >= 0) {
            xin[j + 1] = Xi[kx];
            used[kx] = 1;
        }
        const bool fin = finite_pole(xin[j + 1]);
        double m = 0.0;
        for (int k = 0; k < nb; ++k) {
            sb[k] *= (bnd[k] - sig[j + 1]);
            if (fin) sb[k] /= (1.0 - bnd[k] / xin[j + 1]);
            m = std::max(m, std::abs(sb[k]));
        }
        for (size_t k = 0; k < Xi.size(); ++k) {
            if (used[k] && (int)k == kx) {
                sx[k] = cd(kInf, 0.0);
                continue;
            }
            sx[k] *= (Xi[k] - sig[j + 1]);
            if (fin) sx[k] /= (1.0 - Xi[k] / xin[j + 1]);
        }
        if (m > 0.0 && std::isfinite(m)) {
            for (auto& v : sb) v /= m;
            for (auto& v : sx) v /= m;
        }
    }
    int d = 1;
    std::vector<cd> xi;
    std::vector<double> beta;
    std::vector<cd> dd;
    bool converged = false;
    for (d = 1; d <= dmax; ++d) {
        xi.assign(xin.begin(), xin.begin() + d + 1);
        xi[d] = cd(kInf, 0.0);  // the last pole of the interpolant is infinity
        beta.assign(d + 1, 1.0);
        std::vector<cd> bv(nb, 1.0);
        for (int j = 1; j <= d; ++j) {
            double m = 0.0;
            for (int k = 0; k < nb; ++k) {
                cd g = bv[k] * (bnd[k] - sig[j - 1]);
                if (finite_pole(xi[j])) g /= (1.0 - bnd[k] / xi[j]);
                bv[k] = g;
                m = std::max(m, std::abs(g));
            }
            beta[j] = m;
            for (auto& v : bv) v /= m;
        }
        // d_i^j = e_j^T f_i(H K^{-1}) e_1 (Eq. (nleigsfdd), beta_0 = 1): H lower bidiagonal with the
        // nodes on its diagonal and beta_j below, K with ones and beta_j / xi_j
        LMat Hm(d + 1), Km = lm_eye(d + 1);
        for (int j = 0; j <= d; ++j) Hm(j, j) = sig[j];
        for (int j = 1; j <= d; ++j) {
            Hm(j, j - 1) = beta[j];
            Km(j, j - 1) = finite_pole(xi[j]) ? beta[j] / xi[j] : cd(0.0);
        }
        const LMat Mm = lm_mul(Hm, lm_solve(Km, lm_eye(d + 1)));
        dd.assign((size_t)nt * (d + 1), 0.0);
        for (int i = 0; i < nt; ++i) {
            const LMat Fm = lm_fn(nodes, pool, roots[i], Mm, 0);
            for (int j = 0; j <= d; ++j) dd[i + (size_t)nt * j] = Fm(j, 0);
        }
        double d0 = 0.0, dl = 0.0;
        for (int i = 0; i < nt; ++i) {
            d0 = std::max(d0, std::abs(dd[i]));
            dl = std::max(dl, std::abs(dd[i + (size_t)nt * d]));
        }
        if (dl < tol * d0) {
            converged = true;
            break;
        }
        if (d == dmax) break;
    }
    out->d = d;
    out->converged = converged;
    out->sigma.clear();
    out->xi.clear();
    out->dd.clear();
    for (int j = 0; j <= d; ++j) {
        out->sigma.push_back(to_zd(sig[j]));
        out->xi.push_back(to_zd(xi[j]));
    }
    out->xi[0] = mk(kInf, 0.0);
    out->beta = beta;
    for (auto v : dd) out->dd.push_back(to_zd(v));
    out->nsing = (int)Xi.size();
    return NEP_OK;
}

// ------------------------------------------------------------------ device kernels
constexpr int kNleigsMaxTerms = 8;
constexpr double kNleigsCandidate = 1e-4;  // eta of a Ritz pair worth polishing (fast mode)
constexpr int kNleigsRefine = 2;  // FP64-residual corrections per solve of R_d(sigma), exact mode

struct ExpandCoef {
    zd inv_ds[64];  // 1 / (sigma_{j-1} - shift), j = 1 .. d-1
    zd g[64];       // beta_j / xi_j
    zd e[64];       // beta_j (1 - shift / xi_j)
    zd bsig[64];    // b_j(shift), j = 0 .. d-1
};

// p^{d-1} = 0, p^{j-1} = (v^{j-1} + g_j v^j - e_j p^j) inv_ds_j (j = d-1 .. 1), written to W;
// C[i n + r] = sum_{j<=d-2} dd_i^j p^j + dd_i^d / beta_d v^{d-1}. One thread per row.
__global__ void nleigs_expand_kernel(int n, int d, int nt, const zd* __restrict__ v, zd* __restrict__ W,
                                     zd* __restrict__ C, const ExpandCoef* __restrict__ ec,
                                     const zd* __restrict__ ddc /* nt x (d+1), column d already / beta_d */) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    zd acc[kNleigsMaxTerms];
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i) acc[i] = mk(0.0, 0.0);
    zd vj = v[(int64_t)(d - 1) * n + r];  // v^{d-1}
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i)
        if (i < nt) acc[i] = ddc[i + (int64_t)nt * d] * vj;
    W[(int64_t)(d - 1) * n + r] = mk(0.0, 0.0);
    zd pj = mk(0.0, 0.0);
    for (int j = d - 1; j >= 1; --j) {
        const zd vjm = v[(int64_t)(j - 1) * n + r];
        const zd z = fma_(vjm, ec->g[j], vj);
        const zd p = (z - ec->e[j] * pj) * ec->inv_ds[j];
        W[(int64_t)(j - 1) * n + r] = p;
#pragma unroll
        for (int i = 0; i < kNleigsMaxTerms; ++i)
            if (i < nt) acc[i] = fma_(acc[i], ddc[i + (int64_t)nt * (j - 1)], p);
        pj = p;
        vj = vjm;
    }
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i)
        if (i < nt) C[(int64_t)i * n + r] = acc[i];
}

// The Chebyshev-basis linearisation of P_d(theta) = sum_k C'_k tau_k(theta) (Sec. 4.4): block rows
// -theta u_0 + u_1 = 0, u_{k-1} - 2 theta u_k + u_{k+1} = 0 (1 <= k <= d-2) and the last row
// sum_{k<d} C'_k u_k + C_d (2 theta u_{d-1} - u_{d-2}) = 0, i.e. B v = (v_0, 2 v_1, .., 2 v_{d-2},
// -2 C_d v_{d-1}). The solve (A - sigma B) w = B v: the particular solution p with p_0 = 0,
// p_1 = v_0, p_{k+1} = 2 v_k + 2 sigma p_k - p_{k-1} (k = 1 .. d-2) is written to W, then
// P_d(sigma) w_0 = -sum_i A_i C_i with the per-term combinations
//   C_i = sum_{k<d} c'_ik p_k + c_id (2 sigma p_{d-1} - p_{d-2} + 2 v_{d-1}),
// and w_k = p_k + tau_k(sigma) w_0 (nleigs_combine_kernel). cc: nt x (d+1), c'_i0 = c_i0 / 2.
// One thread per row.
__global__ void cheb_expand_kernel(int n, int d, int nt, const zd* __restrict__ v, zd* __restrict__ W,
                                   zd* __restrict__ C, zd sigma, const zd* __restrict__ cc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    zd acc[kNleigsMaxTerms];
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i) acc[i] = mk(0.0, 0.0);
    zd pm = mk(0.0, 0.0);          // p_{k-1}
    zd pk = v[r];                  // p_1 = v_0
    W[r] = mk(0.0, 0.0);           // p_0
    W[(int64_t)n + r] = pk;
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i)
        if (i < nt) acc[i] = cc[i + (int64_t)nt * 1] * pk;
    const zd two_sigma = mk(2.0 * sigma.re, 2.0 * sigma.im);
    for (int k = 1; k <= d - 2; ++k) {
        const zd vk = v[(int64_t)k * n + r];
        const zd pn = fma_(mk(2.0 * vk.re, 2.0 * vk.im) - pm, two_sigma, pk);  // 2 v_k + 2 sigma p_k - p_{k-1}
        W[(int64_t)(k + 1) * n + r] = pn;
#pragma unroll
        for (int i = 0; i < kNleigsMaxTerms; ++i)
            if (i < nt) acc[i] = fma_(acc[i], cc[i + (int64_t)nt * (k + 1)], pn);
        pm = pk;
        pk = pn;
    }
    // pk = p_{d-1}, pm = p_{d-2}
    const zd vl = v[(int64_t)(d - 1) * n + r];
    const zd tail = fma_(mk(2.0 * vl.re, 2.0 * vl.im) - pm, two_sigma, pk);  // 2 sigma p_{d-1} - p_{d-2} + 2 v_{d-1}
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i)
        if (i < nt) C[(int64_t)i * n + r] = fma_(acc[i], cc[i + (int64_t)nt * d], tail);
}

// out[r] = -sum_e sum_i a_i(r, col e) C[i n + col e]; one warp per row
__global__ void nleigs_spmv_kernel(SplitDev s, const zd* __restrict__ C, zd* __restrict__ out) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= s.n) return;
    const int r = (int)gw;
    zd acc = mk(0.0, 0.0);
    for (int64_t e = s.rowptr[r] + lane; e < s.rowptr[r + 1]; e += 32) {
        const int c = s.col[e];
        for (int i = 0; i < s.nterms; ++i) {
            const zd a = mk(s.val[(int64_t)i * s.nnz + e], s.val_im ? s.val_im[(int64_t)i * s.nnz + e] : 0.0);
            acc = fma_(acc, a, C[(int64_t)i * s.n + c]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) out[r] = mk(-acc.re, -acc.im);
}

// W^j += b_j(shift) u, j = 0 .. d-1
__global__ void nleigs_combine_kernel(int n, int d, const zd* __restrict__ u, zd* __restrict__ W,
                                      const ExpandCoef* __restrict__ ec) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * d) return;
    const int j = (int)(t / n), r = (int)(t % n);
    W[t] = fma_(W[t], ec->bsig[j], u[r]);
}

// h = sqrt(Re nr); H sub-diagonal entry (or hlast) = h; w /= h (w = 0 after a breakdown)
__global__ void nleigs_scale_kernel(int64_t N, zd* __restrict__ w, const zd* __restrict__ nr, zd* __restrict__ hsub) {
    const double h = sqrt(fmax(nr->re, 0.0));
    const double sc = h > 1e-300 ? 1.0 / h : 0.0;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) w[t] = sc * w[t];
    if (t == 0) *hsub = mk(h, 0.0);
}

// Ritz vector of theta_e (one warp per Ritz value, FP64): the upper Hessenberg H - theta I is
// factored with adjacent-row pivoting (an exactly zero pivot stands for eps |H|), three steps of
// inverse iteration from a constant vector follow, and theta becomes the Rayleigh quotient
// s^H H s of the unit vector s. theta comes from the complex64 Hessenberg QR: inverse iteration
// with that shift converges to the FP64 eigenvector at the rate |theta - theta_e| / gap.
__global__ void __launch_bounds__(32) nleigs_ritz_vectors_kernel(int m, const zd* __restrict__ H,
                                                                 zd* __restrict__ theta, zd* __restrict__ S,
                                                                 zd* __restrict__ work, int* __restrict__ pivw) {
    extern __shared__ zd y[];  // m
    const int e = blockIdx.x, lane = threadIdx.x;
    zd* A = work + (int64_t)e * m * m;
    int* pv = pivw + (int64_t)e * m;
    const zd th = theta[e];
    double anorm = 0.0;
    for (int64_t t = lane; t < (int64_t)m * m; t += 32) {
        const int i = (int)(t % m), j = (int)(t / m);
        zd a = i <= j + 1 ? H[t] : mk(0.0, 0.0);
        if (i == j) a = a - th;
        A[t] = a;
        anorm = fmax(anorm, abs1(a));
    }
    for (int o = 16; o > 0; o >>= 1) anorm = fmax(anorm, __shfl_xor_sync(0xffffffffu, anorm, o));
    const double tiny = 1.2e-16 * (anorm > 0.0 ? anorm : 1.0);
    __syncwarp();
    // Hessenberg LU: at column k only rows k and k+1 hold entries on or below the diagonal
    for (int k = 0; k + 1 < m; ++k) {
        const zd a0 = A[k + (int64_t)m * k], a1 = A[k + 1 + (int64_t)m * k];
        const bool sw = abs1(a1) > abs1(a0);
        __syncwarp();
        if (sw)
            for (int j = k + lane; j < m; j += 32) {
                const zd t = A[k + (int64_t)m * j];
                A[k + (int64_t)m * j] = A[k + 1 + (int64_t)m * j];
                A[k + 1 + (int64_t)m * j] = t;
            }
        __syncwarp();
        zd piv = A[k + (int64_t)m * k];
        if (piv.re == 0.0 && piv.im == 0.0) piv = mk(tiny, 0.0);
        const zd lm = cdiv(sw ? a0 : a1, piv);
        for (int j = k + 1 + lane; j < m; j += 32) A[k + 1 + (int64_t)m * j] = fms(A[k + 1 + (int64_t)m * j], lm, A[k + (int64_t)m * j]);
        __syncwarp();
        if (lane == 0) {
            A[k + (int64_t)m * k] = piv;
            A[k + 1 + (int64_t)m * k] = lm;
            pv[k] = sw;
        }
        __syncwarp();
    }
    if (lane == 0) {
        const zd d = A[(m - 1) + (int64_t)m * (m - 1)];
        if (d.re == 0.0 && d.im == 0.0) A[(m - 1) + (int64_t)m * (m - 1)] = mk(tiny, 0.0);
    }
    const double inv_sqrt_m = 1.0 / sqrt((double)m);
    for (int i = lane; i < m; i += 32) y[i] = mk(inv_sqrt_m, 0.0);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
        if (lane == 0)  // forward: the interchanges and multipliers, in order
            for (int k = 0; k + 1 < m; ++k) {
                if (pv[k]) {
                    const zd t = y[k];
                    y[k] = y[k + 1];
                    y[k + 1] = t;
                }
                y[k + 1] = fms(y[k + 1], A[k + 1 + (int64_t)m * k], y[k]);
            }
        __syncwarp();
        for (int k = m - 1; k >= 0; --k) {  // backward with U, by columns
            const zd yk = cdiv(y[k], A[k + (int64_t)m * k]);
            __syncwarp();
            if (lane == 0) y[k] = yk;
            for (int i = lane; i < k; i += 32) y[i] = fms(y[i], A[i + (int64_t)m * k], yk);
            __syncwarp();
        }
        double nn = 0.0;
        for (int i = lane; i < m; i += 32) nn += norm2(y[i]);
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        for (int i = lane; i < m; i += 32) y[i] = sc * y[i];
        __syncwarp();
    }
    // Rayleigh quotient s^H H s (H upper Hessenberg)
    zd rq = mk(0.0, 0.0);
    for (int i = lane; i < m; i += 32) {
        zd hs = mk(0.0, 0.0);
        for (int j = max(0, i - 1); j < m; ++j) hs = fma_(hs, H[i + (int64_t)m * j], y[j]);
        rq = fmac(rq, y[i], hs);
    }
    for (int o = 16; o > 0; o >>= 1) {
        rq.re += __shfl_xor_sync(0xffffffffu, rq.re, o);
        rq.im += __shfl_xor_sync(0xffffffffu, rq.im, o);
    }
    for (int i = lane; i < m; i += 32) S[i + (int64_t)m * e] = y[i];
    if (lane == 0 && isfinite(rq.re) && isfinite(rq.im)) theta[e] = rq;
}

// ---- Krylov-Schur restart with locking, on top of the Arnoldi of Sec. 4.5.3. After a restart the
// projected matrix H (m x m) is no longer Hessenberg: the kept p x p block Q^H H Q (upper triangular:
// Q holds leading Schur vectors), the coupling row p below it, then Hessenberg columns p .. m-1 from
// the continued Arnoldi.

// Ritz vector of theta_e for a general H (one warp per Ritz value, FP64): H - theta I by Gaussian
// elimination with partial pivoting (whole rows swapped; an exactly zero pivot stands for eps |H|),
// three steps of inverse iteration from a constant vector, theta replaced by the Rayleigh quotient
// s^H H s of the unit vector s.
__global__ void __launch_bounds__(32) ks_ritz_vectors_kernel(int m, const zd* __restrict__ H, zd* __restrict__ theta,
                                                             zd* __restrict__ S, zd* __restrict__ work,
                                                             int* __restrict__ pivw) {
    extern __shared__ zd y[];  // m
    const int e = blockIdx.x, lane = threadIdx.x;
    zd* A = work + (int64_t)e * m * m;
    int* pv = pivw + (int64_t)e * m;
    const zd th = theta[e];
    double anorm = 0.0;
    for (int64_t t = lane; t < (int64_t)m * m; t += 32) {
        const int i = (int)(t % m), j = (int)(t / m);
        zd a = H[t];
        if (i == j) a = a - th;
        A[t] = a;
        anorm = fmax(anorm, abs1(a));
    }
    for (int o = 16; o > 0; o >>= 1) anorm = fmax(anorm, __shfl_xor_sync(0xffffffffu, anorm, o));
    const double tiny = 1.2e-16 * (anorm > 0.0 ? anorm : 1.0);
    __syncwarp();
    for (int k = 0; k < m; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + lane; i < m; i += 32) {
            const double a = abs1(A[i + (int64_t)m * k]);
            if (a > best) {
                best = a;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) pv[k] = bi;
        if (bi != k)
            for (int j = lane; j < m; j += 32) {
                const zd t = A[k + (int64_t)m * j];
                A[k + (int64_t)m * j] = A[bi + (int64_t)m * j];
                A[bi + (int64_t)m * j] = t;
            }
        __syncwarp();
        zd piv = A[k + (int64_t)m * k];
        if (piv.re == 0.0 && piv.im == 0.0) piv = mk(tiny, 0.0);
        const zd rp = cdiv(mk(1.0, 0.0), piv);
        __syncwarp();
        if (lane == 0) A[k + (int64_t)m * k] = piv;
        for (int i = k + 1 + lane; i < m; i += 32) A[i + (int64_t)m * k] = A[i + (int64_t)m * k] * rp;
        __syncwarp();
        for (int i = k + 1 + lane; i < m; i += 32) {
            const zd l = A[i + (int64_t)m * k];
            for (int j = k + 1; j < m; ++j) A[i + (int64_t)m * j] = fms(A[i + (int64_t)m * j], l, A[k + (int64_t)m * j]);
        }
        __syncwarp();
    }
    const double inv_sqrt_m = 1.0 / sqrt((double)m);
    for (int i = lane; i < m; i += 32) y[i] = mk(inv_sqrt_m, 0.0);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
        for (int k = 0; k < m; ++k) {  // forward: the interchanges and the unit lower factor
            const int p = pv[k];
            if (p != k && lane == 0) {
                const zd t = y[k];
                y[k] = y[p];
                y[p] = t;
            }
            __syncwarp();
            const zd yk = y[k];
            for (int i = k + 1 + lane; i < m; i += 32) y[i] = fms(y[i], A[i + (int64_t)m * k], yk);
            __syncwarp();
        }
        for (int k = m - 1; k >= 0; --k) {  // backward with U, by columns
            const zd yk = cdiv(y[k], A[k + (int64_t)m * k]);
            __syncwarp();
            if (lane == 0) y[k] = yk;
            for (int i = lane; i < k; i += 32) y[i] = fms(y[i], A[i + (int64_t)m * k], yk);
            __syncwarp();
        }
        double nn = 0.0;
        for (int i = lane; i < m; i += 32) nn += norm2(y[i]);
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        for (int i = lane; i < m; i += 32) y[i] = sc * y[i];
        __syncwarp();
    }
    zd rq = mk(0.0, 0.0);
    for (int i = lane; i < m; i += 32) {
        zd hs = mk(0.0, 0.0);
        for (int j = 0; j < m; ++j) hs = fma_(hs, H[i + (int64_t)m * j], y[j]);
        rq = fmac(rq, y[i], hs);
    }
    for (int o = 16; o > 0; o >>= 1) {
        rq.re += __shfl_xor_sync(0xffffffffu, rq.re, o);
        rq.im += __shfl_xor_sync(0xffffffffu, rq.im, o);
    }
    for (int i = lane; i < m; i += 32) S[i + (int64_t)m * e] = y[i];
    if (lane == 0 && isfinite(rq.re) && isfinite(rq.im)) theta[e] = rq;
}

// res[q] = |b^T s_q|, the residual estimate of the Ritz pair q (unit s_q): b is the row m of the
// (m+1) x m matrix Hf (leading dimension ldh) of the decomposition S V_m = V_{m+1} Hf
__global__ void ks_residual_kernel(int m, int ldh, const zd* __restrict__ Hf, const zd* __restrict__ S,
                                   double* __restrict__ res) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    zd acc = mk(0.0, 0.0);
    for (int j = 0; j < m; ++j) acc = fma_(acc, Hf[m + (int64_t)ldh * j], S[j + (int64_t)m * q]);
    res[q] = sqrt(norm2(acc));
}

// bn[j] = sum_i b_i Q[i, j] for j < p, b the row m of Hf; zero for the nlock locked columns, whose
// coupling to the rest is dropped so that they stay an invariant subspace
__global__ void ks_coupling_kernel(int m, int ldh, int p, int nlock, const zd* __restrict__ Hf,
                                   const zd* __restrict__ Q, zd* __restrict__ bn) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p) return;
    zd acc = mk(0.0, 0.0);
    if (j >= nlock)
        for (int i = 0; i < m; ++i) acc = fma_(acc, Hf[m + (int64_t)ldh * i], Q[i + (int64_t)m * j]);
    bn[j] = acc;
}

// row p of Hf (leading dimension ldh) = bn[0 .. p)
__global__ void ks_set_row_kernel(int p, int ldh, const zd* __restrict__ bn, zd* __restrict__ Hf) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < p) Hf[p + (int64_t)ldh * j] = bn[j];
}

// A = M^H (rows x m, rows >= ncols, zero rows from ncols on): M is the m x ncols matrix whose
// columns are the coefficient blocks g_k^i (column k d + i, leading dimension Mx)
__global__ void ks_blocks_h_kernel(int m, int Mx, int ncols, int rows, const zd* __restrict__ G, zd* __restrict__ A) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * m) return;
    const int r = (int)(t % rows), q = (int)(t / rows);
    A[t] = r < ncols ? conj(G[q + (int64_t)Mx * r]) : mk(0.0, 0.0);
}

// lam = shift + 1/theta; ok = theta != 0 and finite
// lambda = shift + scale / theta for a Ritz value theta of S = (A - sigma B)^{-1} B
__global__ void nleigs_ritz_kernel(int m, const zd* __restrict__ theta, zd shift, zd scale, zd* __restrict__ lam,
                                   int* __restrict__ ok) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const zd t = theta[i];
    const bool nz = (t.re != 0.0 || t.im != 0.0) && isfinite(t.re) && isfinite(t.im);
    lam[i] = nz ? shift + cdiv(scale, t) : mk(0.0, 0.0);
    ok[i] = nz && isfinite(lam[i].re) && isfinite(lam[i].im);
}

__global__ void nleigs_normalize_start_kernel(int64_t N, zd* __restrict__ w, const zd* __restrict__ nr) {
    const double h = sqrt(fmax(nr->re, 0.0));
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) w[t] = (h > 0.0 ? 1.0 / h : 0.0) * w[t];
}

// part[c + nchunks j] = sum over rows of chunk c of conj(V[r + N j]) w[r]; grid (nchunks, K)
__global__ void __launch_bounds__(256) nleigs_dots_kernel(int64_t N, int64_t chunk, const zd* __restrict__ V,
                                                          const zd* __restrict__ w, zd* __restrict__ part) {
    const int c = blockIdx.x, j = blockIdx.y;
    const int64_t r0 = (int64_t)c * chunk, r1 = min(N, r0 + chunk);
    const zd* v = V + (int64_t)j * N;
    zd acc = mk(0.0, 0.0);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) acc = fmac(acc, v[r], w[r]);
    for (int o = 16; o > 0; o >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    __shared__ zd red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        zd t = mk(0.0, 0.0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = t + red[q];
        part[c + (int64_t)gridDim.x * j] = t;
    }
}

// h[j] = sum_c part[c + nchunks j] (fixed order)
__global__ void nleigs_dots_reduce_kernel(int nchunks, int K, const zd* __restrict__ part, zd* __restrict__ h) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    zd t = mk(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) t = t + part[c + (int64_t)nchunks * j];
    h[j] = t;
}

// w[r] -= sum_{j<K} V[r + N j] h[j]; Hcol[j] += h[j] (block 0)
__global__ void __launch_bounds__(256) nleigs_sub_kernel(int64_t N, int K, const zd* __restrict__ V,
                                                         const zd* __restrict__ h, zd* __restrict__ w,
                                                         zd* __restrict__ Hcol) {
    extern __shared__ zd hs[];
    for (int j = threadIdx.x; j < K; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    if (blockIdx.x == 0 && Hcol)
        for (int j = threadIdx.x; j < K; j += blockDim.x) Hcol[j] = Hcol[j] + hs[j];
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    zd acc = w[r];
    for (int j = 0; j < K; ++j) acc = fms(acc, V[r + (int64_t)j * N], hs[j]);
    w[r] = acc;
}


// ---- the compact (TOAR) basis of Sec. 4.5.3: Krylov vectors (I_d (x) U) g with U (n x m) orthonormal,
// growing by one column per step, and coefficient blocks g^i in C^m. Coefficient vectors are stored
// with a fixed stride: block i of vector k at G[k d Mx + i Mx .. + m), zeros beyond m.

// Eq. (nleigs-toar1) on coefficients: pt^{d-1} = 0, pt^{j-1} = (g^{j-1} + g_j g^j - e_j pt^j) inv_ds_j
// (j = d-1 .. 1: the recurrence of nleigs_expand_kernel, acting on U's coordinates), and the per-term
// combinations Cc[t Mx + q] = sum_{j<=d-2} ddc[t, j] pt^j_q + ddc[t, d] g^{d-1}_q, whose images U Cc_t
// enter the split SpMV of Eq. (nleigs-toar2). One thread per coordinate q < m.
__global__ void toar_coef_kernel(int d, int m, int Mx, int nt, const zd* __restrict__ g, zd* __restrict__ pt,
                                 zd* __restrict__ Cc, const ExpandCoef* __restrict__ ec,
                                 const zd* __restrict__ ddc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    zd acc[kNleigsMaxTerms];
    zd gj = g[(int64_t)(d - 1) * Mx + q];
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i) acc[i] = i < nt ? ddc[i + (int64_t)nt * d] * gj : mk(0.0, 0.0);
    pt[(int64_t)(d - 1) * Mx + q] = mk(0.0, 0.0);
    zd pj = mk(0.0, 0.0);
    for (int j = d - 1; j >= 1; --j) {
        const zd gjm = g[(int64_t)(j - 1) * Mx + q];
        const zd z = fma_(gjm, ec->g[j], gj);
        const zd pv = (z - ec->e[j] * pj) * ec->inv_ds[j];
        pt[(int64_t)(j - 1) * Mx + q] = pv;
#pragma unroll
        for (int i = 0; i < kNleigsMaxTerms; ++i)
            if (i < nt) acc[i] = fma_(acc[i], ddc[i + (int64_t)nt * (j - 1)], pv);
        pj = pv;
        gj = gjm;
    }
#pragma unroll
    for (int i = 0; i < kNleigsMaxTerms; ++i)
        if (i < nt) Cc[(int64_t)i * Mx + q] = acc[i];
}

// Eq. (nleigs-toar4): the coefficients of S v in the (possibly extended) basis,
// gn^i = [pt^i ; 0] + b_i(sigma) [h ; rho] (rho only when U grew), zeros beyond mnew.
__global__ void toar_next_kernel(int d, int m, int mnew, int Mx, const zd* __restrict__ pt, const zd* __restrict__ h,
                                 const zd* __restrict__ rho, const ExpandCoef* __restrict__ ec, zd* __restrict__ gn) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)d * Mx) return;
    const int i = (int)(t / Mx), q = (int)(t - (int64_t)i * Mx);
    zd v = mk(0.0, 0.0);
    if (q < m) v = fma_(pt[t], ec->bsig[i], h[q]);
    else if (q == m && mnew > m) v = ec->bsig[i] * (*rho);
    gn[t] = v;
}

// column i of U from block i of the start vector (start of the compact basis); w0 is d x n
__global__ void toar_copy_kernel(int n, const zd* __restrict__ src, zd* __restrict__ dst) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dst[r] = src[r];
}
// the start coefficients: g^i = (h_i ; rho_i) for the Gram-Schmidt of the start blocks
__global__ void toar_start_coef_kernel(int i, int Mx, const zd* __restrict__ h, const zd* __restrict__ rho,
                                       zd* __restrict__ g) {
    const int q = threadIdx.x;
    if (q < i) g[(int64_t)i * Mx + q] = h[q];
    if (q == i) g[(int64_t)i * Mx + q] = *rho;
}

// A block linearisation (A, B) of d blocks of n with its shift-and-invert recurrences: which expand
// kernel applies S = (A - sigma B)^{-1} B up to the solve, the per-term coefficients it combines, the
// combine weights (ec.bsig), the shifted matrix in split form (Fs) and the map from a Ritz value
// theta of S to lambda = lam_shift + lam_scale / theta.
struct KrylovLin {
    int kind = 0;  // 0: rational Newton basis (NLEIGS, Sec. 4.5); 1: Chebyshev basis (Interpol, Sec. 4.4)
    bool toar = false;  // compact basis (Sec. 4.5.3) instead of full (d n)-vectors (kind 0 only)
    int d = 0;
    ExpandCoef ec{};
    std::vector<zd> coef;  // nt x (d+1)
    std::vector<zd> Fs;    // nt
    zd sigma{}, lam_shift{}, lam_scale{};
};
static int krylov_lin_run(const SplitDev& s, const KrylovLin& lin, int kmax, const double* start_host, zd c, double ea,
                          double eb, double eig_tol, bool exact, const KsOpts& ks, NleigsOut* res, cudaStream_t st);

int nleigs_run(const SplitDev& s, const NleigsInterp& it, zd shift, int kmax, const double* start_host, zd c,
               double ea, double eb, double eig_tol, bool exact, NleigsOut* res, cudaStream_t st, bool toar,
               const KsOpts& ks) {
    const int nt = s.nterms, d = it.d;
    if (nt > kNleigsMaxTerms || d < 1 || d > 63 || kmax < 1) return NEP_ERR_ARG;
    KrylovLin lin;
    lin.kind = 0;
    lin.toar = toar && s.n >= d;
    lin.d = d;
    lin.sigma = shift;
    lin.lam_shift = shift;
    lin.lam_scale = mk(1.0, 0.0);
    ExpandCoef& ec = lin.ec;
    std::vector<cd> sig, xi;
    for (auto z : it.sigma) sig.push_back(to_cd(z));
    for (auto z : it.xi) xi.push_back(to_cd(z));
    const cd sh = to_cd(shift);
    for (int j = 1; j <= d - 1; ++j) {
        ec.inv_ds[j] = to_zd(1.0 / (sig[j - 1] - sh));
        const bool fin = finite_pole(xi[j]);
        ec.g[j] = to_zd(fin ? it.beta[j] / xi[j] : cd(0.0));
        ec.e[j] = to_zd(it.beta[j] * (fin ? 1.0 - sh / xi[j] : cd(1.0)));
    }
    std::vector<cd> bs;
    basis_at(sh, sig, xi, it.beta, d, &bs);
    for (int j = 0; j < d; ++j) ec.bsig[j] = to_zd(bs[j]);
    std::vector<zd>& ddc = lin.coef;  // nt x (d+1), column d divided by beta_d
    ddc = it.dd;
    for (int i = 0; i < nt; ++i) ddc[i + (size_t)nt * d] = to_zd(to_cd(ddc[i + (size_t)nt * d]) / it.beta[d]);
    lin.Fs.assign(nt, mk(0.0, 0.0));  // R_d(shift) = sum_i Fs_i A_i
    for (int i = 0; i < nt; ++i) {
        cd acc = 0.0;
        for (int j = 0; j <= d; ++j) acc += bs[j] * to_cd(it.dd[i + (size_t)nt * j]);
        lin.Fs[i] = to_zd(acc);
    }
    return krylov_lin_run(s, lin, kmax, start_host, c, ea, eb, eig_tol, exact, ks, res, st);
}

// Interpol (Sec. 4.4): the Chebyshev coefficients c (nt x (d+1), Eq. (polinterpcoef)) of the f_i on the
// real axis [center - a, center + a] of the region, lambda = a theta + center, and shift-and-invert
// Arnoldi on the Chebyshev-basis linearisation of P_d with the shift sigma (in theta).
int interpol_run(const SplitDev& s, const std::vector<zd>& c, int d, zd sigma, double alpha, double beta, int kmax,
                 const double* start_host, zd center, double ea, double eb, double eig_tol, bool exact, NleigsOut* res,
                 cudaStream_t st, const KsOpts& ks) {
    const int nt = s.nterms;
    if (nt > kNleigsMaxTerms || d < 2 || d > 63 || kmax < 1) return NEP_ERR_ARG;
    KrylovLin lin;
    lin.kind = 1;
    lin.d = d;
    lin.sigma = sigma;
    lin.lam_shift = mk(alpha * sigma.re + beta, alpha * sigma.im);
    lin.lam_scale = mk(alpha, 0.0);
    lin.coef = c;
    for (int i = 0; i < nt; ++i) lin.coef[i] = mk(0.5 * c[i].re, 0.5 * c[i].im);  // C'_0 = C_0 / 2
    // tau_k(sigma), k = 0 .. d, and P_d(sigma) = sum_k c'_ik tau_k(sigma) A_i
    std::vector<cd> tau(d + 1);
    const cd sg = to_cd(sigma);
    tau[0] = 1.0;
    tau[1] = sg;
    for (int k = 1; k < d; ++k) tau[k + 1] = 2.0 * sg * tau[k] - tau[k - 1];
    for (int k = 0; k < d; ++k) lin.ec.bsig[k] = to_zd(tau[k]);
    lin.Fs.assign(nt, mk(0.0, 0.0));
    for (int i = 0; i < nt; ++i) {
        cd acc = 0.0;
        for (int k = 0; k <= d; ++k) acc += tau[k] * to_cd(lin.coef[i + (size_t)nt * k]);
        lin.Fs[i] = to_zd(acc);
    }
    return krylov_lin_run(s, lin, kmax, start_host, center, ea, eb, eig_tol, exact, ks, res, st);
}

static int krylov_lin_run(const SplitDev& s, const KrylovLin& lin, int kmax, const double* start_host, zd c, double ea,
                          double eb, double eig_tol, bool exact, const KsOpts& ks, NleigsOut* res, cudaStream_t st) {
    const int refine = exact ? kNleigsRefine : 0;
    const int n = s.n, nt = s.nterms, d = lin.d;
    const int64_t N = (int64_t)d * n;
    const ExpandCoef& ec = lin.ec;
    const std::vector<zd>& ddc = lin.coef;
    const std::vector<zd>& Fs = lin.Fs;
    const zd shift = lin.lam_shift;
    StreamScratch w(st);
    // device arrays
    ExpandCoef* d_ec = nullptr;
    zd *d_ddc = nullptr, *d_F = nullptr, *tval = nullptr, *V = nullptr, *C = nullptr, *rhs = nullptr, *u = nullptr;
    zd *res_r = nullptr, *Hf = nullptr, *hv = nullptr, *nr = nullptr, *part = nullptr;
    zf *ab = nullptr, *ut = nullptr, *B32 = nullptr;
    double *tnorm = nullptr, *dmax = nullptr, *ymax = nullptr;
    int *ipiv = nullptr, *info = nullptr;
    const int kv = s.kl + s.ku;
    const int64_t chunk = 4096;
    const int nchunks = (int)((N + chunk - 1) / chunk);
    NEP_TRY(w.get(&d_ec, 1));
    NEP_TRY(w.get(&d_ddc, (size_t)nt * (d + 1)));
    NEP_TRY(w.get(&d_F, (size_t)nt));
    NEP_TRY(w.get(&ab, (size_t)n * s.ldab));
    NEP_TRY(w.get(&tval, (size_t)s.nnz));
    NEP_TRY(w.get(&tnorm, 1));
    NEP_TRY(w.get(&ipiv, (size_t)n));
    NEP_TRY(w.get(&info, 1));
    if (band_sweeps_fit(s.kl, s.ku)) NEP_TRY(w.get(&ut, (size_t)n * (kv + 1)));
    NEP_TRY(w.get(&V, (size_t)N * (lin.toar ? 1 : kmax + 1)));
    NEP_TRY(w.get(&C, (size_t)nt * n));
    NEP_TRY(w.get(&rhs, (size_t)n));
    NEP_TRY(w.get(&u, (size_t)n));
    NEP_TRY(w.get(&res_r, (size_t)n));
    NEP_TRY(w.get(&B32, (size_t)n));
    NEP_TRY(w.get(&dmax, 1));
    NEP_TRY(w.get(&ymax, 1));
    const int ldh = kmax + 1;  // Hf: (kmax+1) x kmax, S V_k = V_{k+1} Hf[:k+1, :k]
    NEP_TRY(w.get(&Hf, (size_t)ldh * kmax));
    NEP_TRY(w.get(&hv, (size_t)kmax + 1));
    NEP_TRY(w.get(&nr, 1));
    NEP_TRY(w.get(&part, (size_t)std::max<int64_t>(nchunks, ((int64_t)d * (d + kmax) + chunk - 1) / chunk) * (kmax + 1)));
    NEP_CUDA(cudaMemcpyAsync(d_ec, &ec, sizeof(ec), cudaMemcpyHostToDevice, st));
    NEP_CUDA(cudaMemcpyAsync(d_ddc, ddc.data(), sizeof(zd) * ddc.size(), cudaMemcpyHostToDevice, st));
    NEP_CUDA(cudaMemcpyAsync(d_F, Fs.data(), sizeof(zd) * nt, cudaMemcpyHostToDevice, st));
    NEP_CUDA(cudaMemsetAsync(Hf, 0, sizeof(zd) * (size_t)ldh * kmax, st));
    // R_d(shift) factored once in complex64, its FP64 values kept for the refinement residual
    NEP_TRY(launch_assemble<float>(s, 1, d_F, ab, tnorm, tval, st));
    NEP_TRY(launch_band_lu<float>(s, 1, ab, ipiv, info, nullptr, st));
    if (ut) NEP_TRY(band_transpose_u<float>(s, 1, ab, ut, st));
    // ||x||^2 or x^H y over N entries into out (K = 1)
    auto dots = [&](const zd* Vb, int K, const zd* x, zd* out) -> int {
        nleigs_dots_kernel<<<dim3(nchunks, K), 256, 0, st>>>(N, chunk, Vb, x, part);
        NEP_CHECK_LAUNCH();
        nleigs_dots_reduce_kernel<<<ceil_div(K, 128), 128, 0, st>>>(nchunks, K, part, out);
        NEP_CHECK_LAUNCH();
        return NEP_OK;
    };
    // u = R_d(shift)^{-1} rhs: complex64 solve, then kNleigsRefine FP64-residual corrections
    auto solve = [&]() -> int {
        NEP_TRY(launch_convert_rhs<float>(1, n, 1, rhs, B32, st));
        NEP_TRY(launch_band_solve<float>(s, 1, ab, ut, ipiv, 1, B32, nullptr, st));
        NEP_TRY(launch_widen<float>(1, n, 1, B32, u, st));
        for (int it2 = 0; it2 < refine; ++it2) {
            NEP_TRY(launch_split_residual(s, 1, tval, 1, rhs, u, res_r, nullptr, nullptr, st));
            NEP_TRY(launch_refine_prepare<float>(1, n, 1, res_r, B32, nullptr, st));
            NEP_TRY(launch_band_solve<float>(s, 1, ab, ut, ipiv, 1, B32, nullptr, st));
            NEP_TRY(launch_refine_update<float>(1, n, 1, B32, u, dmax, ymax, nullptr, st));
        }
        return NEP_OK;
    };
    // compact basis (Sec. 4.5.3): U, the coefficient vectors Gc (stride d Mx), their Hessenberg matrix
    const int Mx = d + kmax;
    zd *U = nullptr, *Gc = nullptr, *pt = nullptr, *Cc = nullptr, *hacc = nullptr, *hv2 = nullptr, *partn = nullptr;
    zd *rho = nullptr, *nr0 = nullptr;
    int m_cur = 0;
    const int nchunks_n = (int)((n + chunk - 1) / chunk);
    const int64_t NG = (int64_t)d * Mx;
    const int nchunks_g = (int)((NG + chunk - 1) / chunk);
    auto dots_n = [&](const zd* Vb, int K, const zd* x, zd* out) -> int {  // over n entries
        nleigs_dots_kernel<<<dim3(nchunks_n, K), 256, 0, st>>>(n, chunk, Vb, x, partn);
        NEP_CHECK_LAUNCH();
        nleigs_dots_reduce_kernel<<<ceil_div(K, 128), 128, 0, st>>>(nchunks_n, K, partn, out);
        NEP_CHECK_LAUNCH();
        return NEP_OK;
    };
    auto dots_g = [&](const zd* Vb, int K, const zd* x, zd* out) -> int {  // over d Mx coefficient entries
        nleigs_dots_kernel<<<dim3(nchunks_g, K), 256, 0, st>>>(NG, chunk, Vb, x, part);
        NEP_CHECK_LAUNCH();
        nleigs_dots_reduce_kernel<<<ceil_div(K, 128), 128, 0, st>>>(nchunks_g, K, part, out);
        NEP_CHECK_LAUNCH();
        return NEP_OK;
    };
    // u (n) orthogonalised against the m columns of U twice into the column slot m of U; the
    // coefficients accumulate in hacc, rho = its remaining norm; returns whether U grew (not a breakdown)
    std::vector<double> hp(4, 0.0);
    auto extend = [&](const zd* u, int m, bool* grew) -> int {
        zd* col = U + (int64_t)m * n;
        toar_copy_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, u, col);
        NEP_CHECK_LAUNCH();
        NEP_TRY(dots_n(col, 1, col, nr0));
        NEP_CUDA(cudaMemsetAsync(hacc, 0, sizeof(zd) * Mx, st));
        for (int pass = 0; pass < 2 && m > 0; ++pass) {
            NEP_TRY(dots_n(U, m, col, hv2));
            nleigs_sub_kernel<<<ceil_div(n, 256), 256, sizeof(zd) * m, st>>>(n, m, U, hv2, col, hacc);
            NEP_CHECK_LAUNCH();
        }
        NEP_TRY(dots_n(col, 1, col, nr));
        nleigs_scale_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, col, nr, rho);
        NEP_CHECK_LAUNCH();
        NEP_CUDA(cudaMemcpyAsync(hp.data(), nr0, sizeof(double), cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaMemcpyAsync(hp.data() + 2, rho, sizeof(double), cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaStreamSynchronize(st));
        *grew = hp[2] > 64 * 2.220446049250313e-16 * std::sqrt(std::max(hp[0], 0.0)) && hp[2] > 0.0;
        return NEP_OK;
    };
    if (lin.toar) {
        NEP_TRY(w.get(&U, (size_t)n * (Mx + 1)));
        NEP_TRY(w.get(&Gc, (size_t)NG * (kmax + 1)));
        NEP_TRY(w.get(&pt, (size_t)NG));
        NEP_TRY(w.get(&Cc, (size_t)nt * Mx));
        NEP_TRY(w.get(&hacc, (size_t)Mx));
        NEP_TRY(w.get(&hv2, (size_t)Mx));
        NEP_TRY(w.get(&partn, (size_t)nchunks_n * (Mx + 1)));
        NEP_TRY(w.get(&rho, 1));
        NEP_TRY(w.get(&nr0, 1));
        NEP_CUDA(cudaMemsetAsync(Gc, 0, sizeof(zd) * (size_t)NG * (kmax + 1), st));
        // start: the d blocks of the start vector by Gram-Schmidt into U, their coordinates into G_0
        zd* w0 = V;  // the start vector's staging (d blocks of n), the full basis is not used
        NEP_CUDA(cudaMemcpyAsync(w0, start_host, sizeof(zd) * (size_t)N, cudaMemcpyHostToDevice, st));
        for (int i = 0; i < d; ++i) {
            bool grew = false;
            NEP_TRY(extend(w0 + (int64_t)i * n, m_cur, &grew));
            if (!grew) { set_error("nleigs: start blocks linearly dependent"); return NEP_ERR_INTERNAL; }
            toar_start_coef_kernel<<<1, 64, 0, st>>>(i, Mx, hacc, rho, Gc);
            NEP_CHECK_LAUNCH();
            ++m_cur;
        }
        NEP_TRY(dots_g(Gc, 1, Gc, nr));
        nleigs_normalize_start_kernel<<<ceil_div(NG, 256), 256, 0, st>>>(NG, Gc, nr);
        NEP_CHECK_LAUNCH();
    } else {
        // start vector, unit 2-norm
        NEP_CUDA(cudaMemcpyAsync(V, start_host, sizeof(zd) * (size_t)N, cudaMemcpyHostToDevice, st));
        NEP_TRY(dots(V, 1, V, nr));
        nleigs_normalize_start_kernel<<<ceil_div(N, 256), 256, 0, st>>>(N, V, nr);
        NEP_CHECK_LAUNCH();
    }
    // Arnoldi step k: the next Krylov vector from vector k, orthogonalised against vectors 0 .. k
    // into column k of Hf (its subdiagonal entry included)
    auto step = [&](int k) -> int {
        zd* Hcol = Hf + (int64_t)ldh * k;
        if (lin.toar) {
            const zd* gk = Gc + (int64_t)k * NG;
            zd* gn = Gc + (int64_t)(k + 1) * NG;
            toar_coef_kernel<<<ceil_div(m_cur, 128), 128, 0, st>>>(d, m_cur, Mx, nt, gk, pt, Cc, d_ec, d_ddc);
            NEP_CHECK_LAUNCH();
            NEP_TRY(zgemm(n, nt, m_cur, 0, U, n, Cc, Mx, C, n, nullptr, 0, st));  // C_t = U Cc_t
            nleigs_spmv_kernel<<<ceil_div((int64_t)n * 32, 256), 256, 0, st>>>(s, C, rhs);
            NEP_CHECK_LAUNCH();
            NEP_TRY(solve());  // y^0 = R_d(shift)^{-1} rhs in u (Eq. (nleigs-toar2))
            bool grew = false;
            NEP_TRY(extend(u, m_cur, &grew));  // Eq. (nleigs-toar3)
            const int mnew = grew ? m_cur + 1 : m_cur;
            toar_next_kernel<<<ceil_div(NG, 256), 256, 0, st>>>(d, m_cur, mnew, Mx, pt, hacc, rho, d_ec, gn);
            NEP_CHECK_LAUNCH();
            m_cur = mnew;
            // Arnoldi on the coefficient vectors, classical Gram-Schmidt twice
            for (int pass = 0; pass < 2; ++pass) {
                NEP_TRY(dots_g(Gc, k + 1, gn, hv));
                nleigs_sub_kernel<<<ceil_div(NG, 256), 256, sizeof(zd) * (k + 1), st>>>(NG, k + 1, Gc, hv, gn, Hcol);
                NEP_CHECK_LAUNCH();
            }
            NEP_TRY(dots_g(gn, 1, gn, nr));
            nleigs_scale_kernel<<<ceil_div(NG, 256), 256, 0, st>>>(NG, gn, nr, Hcol + k + 1);
            NEP_CHECK_LAUNCH();
            return NEP_OK;
        }
        const zd* vk = V + (int64_t)k * N;
        zd* wk = V + (int64_t)(k + 1) * N;
        if (lin.kind == 0)
            nleigs_expand_kernel<<<ceil_div(n, 128), 128, 0, st>>>(n, d, nt, vk, wk, C, d_ec, d_ddc);
        else
            cheb_expand_kernel<<<ceil_div(n, 128), 128, 0, st>>>(n, d, nt, vk, wk, C, lin.sigma, d_ddc);
        NEP_CHECK_LAUNCH();
        nleigs_spmv_kernel<<<ceil_div((int64_t)n * 32, 256), 256, 0, st>>>(s, C, rhs);
        NEP_CHECK_LAUNCH();
        NEP_TRY(solve());
        nleigs_combine_kernel<<<ceil_div(N, 256), 256, 0, st>>>(n, d, u, wk, d_ec);
        NEP_CHECK_LAUNCH();
        for (int pass = 0; pass < 2; ++pass) {
            NEP_TRY(dots(V, k + 1, wk, hv));
            nleigs_sub_kernel<<<ceil_div(N, 256), 256, sizeof(zd) * (k + 1), st>>>(N, k + 1, V, hv, wk, Hcol);
            NEP_CHECK_LAUNCH();
        }
        NEP_TRY(dots(wk, 1, wk, nr));
        nleigs_scale_kernel<<<ceil_div(N, 256), 256, 0, st>>>(N, wk, nr, Hcol + k + 1);
        NEP_CHECK_LAUNCH();
        return NEP_OK;
    };
    // Ritz pairs of H = Hf[:m, :m] and the restart work arrays
    const int m = kmax;
    zd *theta = nullptr, *S = nullptr, *lam = nullptr, *X = nullptr, *G = nullptr, *Hc = nullptr;
    double* eta = nullptr;
    int *status = nullptr, *ok = nullptr, *order = nullptr;
    zd *gbuf = nullptr, *rwork = nullptr;
    int* rpiv = nullptr;
    NEP_TRY(w.get(&theta, m));
    NEP_TRY(w.get(&S, (size_t)m * m));
    NEP_TRY(w.get(&Hc, (size_t)m * m));
    NEP_TRY(w.get(&lam, m));
    NEP_TRY(w.get(&X, (size_t)n * m));
    NEP_TRY(w.get(&G, (size_t)m * m));
    NEP_TRY(w.get(&eta, m));
    NEP_TRY(w.get(&status, 1));
    NEP_TRY(w.get(&ok, m));
    NEP_TRY(w.get(&order, m + 1));
    NEP_TRY(w.get(&gbuf, (size_t)m * (m + 1) + m));  // complex64 elements fit twice over
    NEP_TRY(w.get(&rwork, (size_t)m * m * m));
    NEP_TRY(w.get(&rpiv, (size_t)m * m));
    double* kres = nullptr;
    int* ksel = nullptr;
    zd *Tq = nullptr, *Zq = nullptr, *sgbuf = nullptr, *bn = nullptr, *tmp = nullptr;
    size_t tmp_elems = 0;
    if (ks.max_restarts > 0) {
        NEP_TRY(w.get(&kres, m));
        NEP_TRY(w.get(&ksel, m));
        NEP_TRY(w.get(&Tq, (size_t)m * m));
        NEP_TRY(w.get(&Zq, (size_t)m * m));
        NEP_TRY(w.get(&sgbuf, (size_t)2 * m * (m + 1) + m));
        NEP_TRY(w.get(&bn, m));
        const int64_t rows_max = lin.toar ? std::max<int64_t>(n, NG) : N;
        tmp_elems = (size_t)std::min<int64_t>(rows_max * (lin.toar ? Mx : m), (int64_t)1 << 22);
        tmp_elems = std::max<size_t>(tmp_elems, (size_t)(lin.toar ? Mx : m));
        NEP_TRY(w.get(&tmp, tmp_elems));
    }
    // X[:, :kout] = X[:, :kin] Qm (rows x kin, leading dimension ld; Qm kin x kout, kout <= kin),
    // in row chunks through tmp
    auto right_mul = [&](zd* Xb, int64_t ld, int64_t rows, int kin, const zd* Qm, int kout) -> int {
        const int64_t R = std::max<int64_t>(1, (int64_t)tmp_elems / kout);
        for (int64_t r0 = 0; r0 < rows; r0 += R) {
            const int rr = (int)std::min<int64_t>(R, rows - r0);
            NEP_TRY(zgemm(rr, kout, kin, 0, Xb + r0, (int)ld, Qm, kin, tmp, rr, nullptr, 0, st));
            NEP_CUDA(cudaMemcpy2DAsync(Xb + r0, sizeof(zd) * ld, tmp, sizeof(zd) * rr, sizeof(zd) * rr, kout,
                                       cudaMemcpyDeviceToDevice, st));
        }
        return NEP_OK;
    };
    // the compact basis after a restart to p + 1 vectors: U <- U Q_r and the coefficients <- Q_r^H
    // (coefficients), Q_r an orthonormal basis of the range of the m_cur x d (p+1) matrix of all
    // coefficient blocks, from QR with column pivoting stopped at a relative Frobenius mass of 1e-13;
    // at most d + p columns are kept (the blocks of p + 1 vectors of a Krylov subspace span at most
    // d + p directions, Sec. 4.5.3)
    zd *Ac = nullptr, *Gt = nullptr, *Qr = nullptr, *qtau = nullptr;
    double* qn2 = nullptr;
    int *qperm = nullptr, *qsteps = nullptr, *qerr = nullptr;
    unsigned* qbar = nullptr;
    auto compress = [&](int p) -> int {
        const int ncols = d * (p + 1);
        if (!Ac) {
            const size_t cmax = (size_t)d * (kmax + 1);
            NEP_TRY(w.get(&Ac, (size_t)Mx * cmax));
            NEP_TRY(w.get(&Gt, (size_t)Mx * cmax));
            NEP_TRY(w.get(&Qr, (size_t)Mx * Mx));
            NEP_TRY(w.get(&qtau, (size_t)Mx));
            NEP_TRY(w.get(&qn2, cmax));
            NEP_TRY(w.get(&qperm, cmax));
            NEP_TRY(w.get(&qsteps, 1));
            NEP_TRY(w.get(&qerr, 1));
            NEP_TRY(w.get(&qbar, 2));
        }
        NEP_CUDA(cudaMemcpy2DAsync(Ac, sizeof(zd) * m_cur, Gc, sizeof(zd) * Mx, sizeof(zd) * m_cur, ncols,
                                   cudaMemcpyDeviceToDevice, st));
        int r = 0;
        NEP_TRY(qr_range_basis(m_cur, ncols, Ac, Qr, d + p, 1e-13, qtau, qperm, qn2, qsteps, qbar, qerr, &r, st));
        NEP_TRY(right_mul(U, n, n, m_cur, Qr, r));
        NEP_TRY(zgemm(r, ncols, m_cur, 1, Qr, m_cur, Gc, Mx, Gt, r, nullptr, 0, st));
        NEP_CUDA(cudaMemsetAsync(Gc, 0, sizeof(zd) * (size_t)ncols * Mx, st));
        NEP_CUDA(cudaMemcpy2DAsync(Gc, sizeof(zd) * Mx, Gt, sizeof(zd) * r, sizeof(zd) * r, ncols,
                                   cudaMemcpyDeviceToDevice, st));
        m_cur = r;
        return NEP_OK;
    };
    int k0 = 0, restarts = 0, total_steps = 0;
    std::vector<zd> th_h(m);
    std::vector<double> res_h(m);
    for (;;) {
        for (int k = k0; k < kmax; ++k) {
            NEP_TRY(step(k));
            ++total_steps;
        }
        // Ritz values: QR after a Hessenberg reduction, then FP64 inverse iteration and Rayleigh
        // quotients (adjacent-row pivoting while H is still Hessenberg). Without restarts the QR runs
        // in complex64; with them it is the FP64 Schur form H = Z T Z^H that the restart reorders (in
        // FP64 also because the locked block's entries below the diagonal, zero up to rounding, can
        // lie below 1e-20 |H|, whose squares FP32 cannot hold)
        NEP_CUDA(cudaMemcpy2DAsync(Hc, sizeof(zd) * m, Hf, sizeof(zd) * ldh, sizeof(zd) * m, m,
                                   cudaMemcpyDeviceToDevice, st));
        if (ks.max_restarts > 0) NEP_TRY(launch_ks_schur(m, Hc, theta, Tq, Zq, status, sgbuf, st));
        else NEP_TRY(small_eig_fast<float>(m, Hc, theta, nullptr, status, gbuf, st));
        if (restarts == 0)
            nleigs_ritz_vectors_kernel<<<m, 32, sizeof(zd) * m, st>>>(m, Hc, theta, S, rwork, rpiv);
        else
            ks_ritz_vectors_kernel<<<m, 32, sizeof(zd) * m, st>>>(m, Hc, theta, S, rwork, rpiv);
        NEP_CHECK_LAUNCH();
        if (restarts >= ks.max_restarts) break;
        ks_residual_kernel<<<ceil_div(m, 128), 128, 0, st>>>(m, ldh, Hf, S, kres);
        NEP_CHECK_LAUNCH();
        NEP_CUDA(cudaMemcpyAsync(th_h.data(), theta, sizeof(zd) * m, cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaMemcpyAsync(res_h.data(), kres, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaStreamSynchronize(st));
        // wanted: lambda = lam_shift + lam_scale / theta strictly inside the region; converged:
        // residual estimate |b^T s| <= tol |theta|
        std::vector<int> conv, rest, others;
        for (int q = 0; q < m; ++q) {
            const cd t = to_cd(th_h[q]);
            bool want = false;
            if (std::abs(t) > 0.0 && std::isfinite(t.real()) && std::isfinite(t.imag())) {
                const cd l = to_cd(lin.lam_shift) + to_cd(lin.lam_scale) / t;
                const double dr = (l.real() - c.re) / ea, di = (l.imag() - c.im) / eb;
                want = dr * dr + di * di < 1.0;
            }
            if (want && res_h[q] <= ks.tol * std::abs(t)) conv.push_back(q);
            else if (want) rest.push_back(q);
            else others.push_back(q);
        }
        if (ks.nev > 0 ? (int)conv.size() >= ks.nev : (conv.size() + rest.size() > 0 && rest.empty())) break;
        auto by_size = [&](std::vector<int>& v) {
            std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return std::abs(to_cd(th_h[a])) > std::abs(to_cd(th_h[b])); });
        };
        by_size(conv);
        by_size(rest);
        by_size(others);
        const int nconv = (int)conv.size();
        const int p = std::min(m - 1, std::max(ks.keep, nconv + 1));
        std::vector<int> sel(conv);
        sel.insert(sel.end(), rest.begin(), rest.end());
        sel.insert(sel.end(), others.begin(), others.end());
        sel.resize(p);
        NEP_CUDA(cudaMemcpyAsync(ksel, sel.data(), sizeof(int) * p, cudaMemcpyHostToDevice, st));
        // the kept Ritz values to the front of the Schur form: Q = Z[:, :p] spans their invariant
        // subspace, H <- T[:p, :p] = Q^H H Q, the coupling row b^T Q with the locked entries zeroed
        NEP_TRY(launch_ks_reorder(m, p, ksel, Tq, Zq, st));
        const int pk = p, nlock = nconv;
        const zd* Qk = Zq;
        ks_coupling_kernel<<<ceil_div(pk, 128), 128, 0, st>>>(m, ldh, pk, nlock, Hf, Qk, bn);
        NEP_CHECK_LAUNCH();
        // basis: vectors 0 .. pk-1 <- V_m Q, vector pk <- vector m
        if (lin.toar) {
            NEP_TRY(right_mul(Gc, NG, NG, m, Qk, pk));
            NEP_CUDA(cudaMemcpyAsync(Gc + (int64_t)pk * NG, Gc + (int64_t)m * NG, sizeof(zd) * NG,
                                     cudaMemcpyDeviceToDevice, st));
            NEP_TRY(compress(pk));
        } else {
            NEP_TRY(right_mul(V, N, N, m, Qk, pk));
            NEP_CUDA(cudaMemcpyAsync(V + (int64_t)pk * N, V + (int64_t)m * N, sizeof(zd) * N,
                                     cudaMemcpyDeviceToDevice, st));
        }
        NEP_CUDA(cudaMemsetAsync(Hf, 0, sizeof(zd) * (size_t)ldh * kmax, st));
        NEP_CUDA(cudaMemcpy2DAsync(Hf, sizeof(zd) * ldh, Tq, sizeof(zd) * m, sizeof(zd) * pk, pk,
                                   cudaMemcpyDeviceToDevice, st));
        ks_set_row_kernel<<<ceil_div(pk, 128), 128, 0, st>>>(pk, ldh, bn, Hf);
        NEP_CHECK_LAUNCH();
        k0 = pk;
        ++restarts;
    }
    nleigs_ritz_kernel<<<ceil_div(m, 128), 128, 0, st>>>(m, theta, shift, lin.lam_scale, lam, ok);
    NEP_CHECK_LAUNCH();
    if (lin.toar) {
        // x = first block of the Ritz vector = U (G^0 S), G^0 the coordinates of block 0
        zd* Z = nullptr;
        NEP_TRY(w.get(&Z, (size_t)Mx * m));
        NEP_TRY(zgemm(m_cur, m, m, 0, Gc, (int)NG, S, m, Z, m_cur, nullptr, 0, st));
        NEP_TRY(zgemm(n, m, m_cur, 0, U, n, Z, m_cur, X, n, nullptr, 0, st));
    } else {
        NEP_TRY(zgemm(n, m, m, 0, V, (int)N, S, m, X, n, nullptr, 0, st));
    }
    NEP_TRY(launch_normalize_columns(n, m, X, 1, nullptr, st));
    NEP_TRY(launch_eta(s, m, lam, X, eta, st));
    if (!exact) {
        // the Arnoldi ran on complex64 solves: Ritz pairs inside the region that converged to that
        // level (eta <= kNleigsCandidate) are polished by residual inverse iteration (FP64
        // residuals) to tol 1e-13 before the acceptance test
        std::vector<zd> lc(m);
        std::vector<double> ec(m);
        std::vector<int> okc(m);
        NEP_CUDA(cudaMemcpyAsync(lc.data(), lam, sizeof(zd) * m, cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaMemcpyAsync(ec.data(), eta, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaMemcpyAsync(okc.data(), ok, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaStreamSynchronize(st));
        std::vector<int> idx;
        for (int i = 0; i < m; ++i) {
            const double dr = (lc[i].re - c.re) / ea, di = (lc[i].im - c.im) / eb;
            if (okc[i] && dr * dr + di * di < 1.0 && ec[i] <= kNleigsCandidate) idx.push_back(i);
        }
        const int P = (int)idx.size();
        if (P > 0) {
            int *didx = nullptr, *pits = nullptr;
            zd *plam = nullptr, *pX = nullptr;
            double* peta = nullptr;
            NEP_TRY(w.get(&didx, P));
            NEP_TRY(w.get(&pits, P));
            NEP_TRY(w.get(&plam, P));
            NEP_TRY(w.get(&pX, (size_t)n * P));
            NEP_TRY(w.get(&peta, P));
            NEP_CUDA(cudaMemcpyAsync(didx, idx.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
            NEP_TRY(launch_rii_move(n, P, didx, lam, X, eta, plam, pX, peta, 0, st));
            int its_max = 0;
            NEP_TRY(rii_polish<float>(s, P, plam, pX, peta, pits, 1e-13, 10, &its_max, st));
            NEP_TRY(launch_rii_move(n, P, didx, lam, X, eta, plam, pX, peta, 1, st));
            res->polished = P;
            res->polish_its = its_max;
        }
    }
    NEP_TRY(zgemm(m, m, n, 1, X, n, X, n, G, m, nullptr, 0, st));
    NEP_TRY(launch_select(m, lam, eta, ok, G, c, ea, eb, eig_tol, order, st));
    std::vector<int> ord(m + 1);
    std::vector<zd> lh(m);
    std::vector<double> eh(m);
    NEP_CUDA(cudaMemcpyAsync(ord.data(), order, sizeof(int) * (m + 1), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaMemcpyAsync(lh.data(), lam, sizeof(zd) * m, cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaMemcpyAsync(eh.data(), eta, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    const int nc = std::max(0, std::min(ord[0], m));
    res->lam.clear();
    res->eta.clear();
    res->X.assign((size_t)n * nc, mk(0.0, 0.0));
    for (int q = 0; q < nc; ++q) {
        const int i = ord[1 + q];
        res->lam.push_back(lh[i]);
        res->eta.push_back(eh[i]);
        NEP_CUDA(cudaMemcpyAsync(res->X.data() + (size_t)n * q, X + (size_t)n * i, sizeof(zd) * n,
                                 cudaMemcpyDeviceToHost, st));
    }
    // all Ritz values (diagnostics)
    res->ritz.assign(lh.begin(), lh.end());
    NEP_CUDA(cudaStreamSynchronize(st));
    int info_h = 0;
    NEP_CUDA(cudaMemcpy(&info_h, info, sizeof(int), cudaMemcpyDeviceToHost));
    res->lu_info = info_h;
    res->steps = total_steps;
    res->restarts = restarts;
    return NEP_OK;
}

}  // namespace nep
