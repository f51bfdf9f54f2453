// Host side of the C ABI: operator construction (split form, Sec. 2 Eq. (split); the
// NEPSetSplitOperator interface of Sec. 3.2.2), region checks, quadrature nodes and
// coefficients, the device-resident plan that runs the whole contour-integral pass, and
// result objects. Every numerical step after the coefficient table runs in the CUDA
// kernels of this library; the host only sizes launches and moves small scalars.
#include <cstdarg>
#include <cstring>
#include <complex>
#include <atomic>
#include <mutex>
#include <set>
#include <map>
#include <tuple>
#include <vector>

#include "nep_common.cuh"

namespace nep {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static std::atomic<long long> g_wait_limit{1ll << 24};
long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? NEP_ERR_NOMEM : NEP_ERR_CUDA;
}

// When g_dry is set, allocations are only counted (plan footprint estimates for admission).
static thread_local bool g_dry = false;
static thread_local size_t g_dry_bytes = 0;

template <typename T>
static int dalloc(T** p, size_t count, cudaStream_t st) {
    *p = nullptr;
    if (count == 0) count = 1;
    const size_t bytes = (sizeof(T) * count + 255) / 256 * 256;
    if (g_dry) {
        g_dry_bytes += bytes;
        return NEP_OK;
    }
    NEP_CUDA(cudaMallocAsync((void**)p, sizeof(T) * count, st));
    return NEP_OK;
}
static int dalloc_raw(void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (g_dry) {
        g_dry_bytes += (bytes + 255) / 256 * 256;
        return NEP_OK;
    }
    NEP_CUDA(cudaMallocAsync(p, bytes, st));
    return NEP_OK;
}

static void configure_pool_once() {
    static std::once_flag flag;
    std::call_once(flag, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        uint64_t thr = UINT64_MAX;  // keep freed blocks cached in this process for reuse by later plans
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    });
}

}  // namespace nep

int nep::smem_optin_bytes() {
    static const int v = [] {
        int dev = 0, b = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || b <= 0)
            b = 227 * 1024;
        return b;
    }();
    return v;
}

namespace {
std::mutex g_smem_mu;
std::set<std::pair<int, const void*>> g_smem_raised;
}  // namespace

bool nep::smem_limit_raised(const void* fn) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_smem_mu);
    return g_smem_raised.count({dev, fn}) != 0;
}

void nep::smem_limit_mark(const void* fn) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_smem_mu);
    g_smem_raised.insert({dev, fn});
}

using namespace nep;

// ============================================================================ split operator
// A term whose function the host supplies (NEP_FN_CALLBACK, NEP_FN_TABLE): never evaluated on the device.
struct ExtTerm {
    int kind = -1;  // -1: built-in (a device function tree)
    nep_fn_eval_t eval = nullptr;
    void* ctx = nullptr;
    std::vector<zd> table;
};

struct nep_split {
    int n = 0, nterms = 0, kl = 0, ku = 0, ldab = 0;
    int64_t nnz = 0;
    bool complex_vals = false;
    std::vector<ExtTerm> ext;  // per term
    bool has_ext = false;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> val, val_im;
    std::vector<double> norms, norms1;
    // the union pattern by columns: entries colptr[c] .. colptr[c+1]-1 of column c, in
    // increasing row order, are union-pattern entry cidx[k] in row crow[k]
    std::vector<int64_t> colptr, cidx;
    std::vector<int32_t> crow;
    std::vector<FnNode> nodes;
    std::vector<zd> coef;
    std::vector<int> roots;
    // device copies
    int64_t* d_rowptr = nullptr;
    int32_t* d_col = nullptr;
    double* d_val = nullptr;
    double* d_val_im = nullptr;
    double* d_norms = nullptr;
    double* d_norms1 = nullptr;
    int64_t* d_colptr = nullptr;
    int64_t* d_cidx = nullptr;
    int32_t* d_crow = nullptr;
    FnNode* d_nodes = nullptr;
    zd* d_coef = nullptr;
    int* d_roots = nullptr;
    int device = 0;
    SplitDev dev() const {
        SplitDev s;
        s.n = n;
        s.nterms = nterms;
        s.kl = kl;
        s.ku = ku;
        s.ldab = ldab;
        s.nnz = nnz;
        s.rowptr = d_rowptr;
        s.col = d_col;
        s.val = d_val;
        s.val_im = complex_vals ? d_val_im : nullptr;
        s.norms = d_norms;
        s.norms1 = d_norms1;
        s.colptr = d_colptr;
        s.cidx = d_cidx;
        s.crow = d_crow;
        s.fn_nodes = d_nodes;
        s.fn_coef = d_coef;
        s.fn_root = d_roots;
        return s;
    }
};

static int flatten_fn(nep_split* h, const nep_fn* f, int depth) {
    if (!f) { set_error("null function description"); return -1; }
    if (depth > 16) { set_error("function tree deeper than 16 levels"); return -1; }
    FnNode nd;
    memset(&nd, 0, sizeof(nd));
    nd.kind = f->kind;
    nd.op = f->op;
    nd.alpha = mk(f->alpha_re, f->alpha_im);
    nd.beta = mk(f->beta_re, f->beta_im);
    nd.shift = mk(f->shift_re, f->shift_im);
    nd.a = nd.b = -1;
    if (f->kind == NEP_FN_RATIONAL) {
        if (f->nnum < 1 || !f->num) { set_error("rational function needs at least one numerator coefficient"); return -1; }
        if (f->nden < 0 || (f->nden > 0 && !f->den)) { set_error("bad denominator"); return -1; }
        nd.num_off = (int)h->coef.size();
        nd.num_len = f->nnum;
        for (int i = 0; i < f->nnum; ++i) h->coef.push_back(mk(f->num[2 * i], f->num[2 * i + 1]));
        nd.den_off = (int)h->coef.size();
        nd.den_len = f->nden;
        for (int i = 0; i < f->nden; ++i) h->coef.push_back(mk(f->den[2 * i], f->den[2 * i + 1]));
    } else if (f->kind == NEP_FN_EXP || f->kind == NEP_FN_SQRT) {
    } else if (f->kind == NEP_FN_CALLBACK || f->kind == NEP_FN_TABLE) {
        if (depth > 0) { set_error("callback and table functions are allowed only at the top level of a term"); return -1; }
    } else if (f->kind == NEP_FN_COMBINE) {
        if (f->op < NEP_OP_ADD || f->op > NEP_OP_COMPOSE) { set_error("bad combine op %d", f->op); return -1; }
        const int self = (int)h->nodes.size();
        h->nodes.push_back(nd);
        const int a = flatten_fn(h, f->a, depth + 1);
        if (a < 0) return -1;
        const int b = flatten_fn(h, f->b, depth + 1);
        if (b < 0) return -1;
        h->nodes[self].a = a;
        h->nodes[self].b = b;
        return self;
    } else {
        set_error("unknown function kind %d", f->kind);
        return -1;
    }
    h->nodes.push_back(nd);
    return (int)h->nodes.size() - 1;
}

static void free_split_device(nep_split* h) {
    void* bufs[] = {h->d_rowptr, h->d_col, h->d_val, h->d_val_im, h->d_norms, h->d_norms1,
                    h->d_colptr, h->d_cidx, h->d_crow, h->d_nodes, h->d_coef, h->d_roots};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, 0);
}

// the split's arrays come from the stream-ordered pool on the legacy stream (the caller synchronises
// it once after all uploads), so that destroying a split frees them without the device-wide
// synchronisation of cudaFree
template <typename T>
static int upload(T** d, const std::vector<T>& v) {
    const size_t bytes = sizeof(T) * (v.size() ? v.size() : 1);
    NEP_CUDA(cudaMallocAsync((void**)d, bytes, 0));
    if (!v.empty()) NEP_CUDA(cudaMemcpyAsync(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, 0));
    return NEP_OK;
}

extern "C" int nep_create_split(int32_t n, int32_t nterms, const nep_csr* A, const nep_fn* f, nep_split_t* out) {
    if (!out) { set_error("out is NULL"); return NEP_ERR_ARG; }
    *out = nullptr;
    if (n < 1 || nterms < 1 || nterms > 32 || !A || !f) {
        set_error("nep_create_split: need n >= 1, 1 <= nterms <= 32 and non-NULL A, f");
        return NEP_ERR_ARG;
    }
    for (int i = 0; i < nterms; ++i) {
        const nep_csr& c = A[i];
        if (c.n_rows != n || c.n_cols != n || !c.rowptr || !c.col || !c.val_re) {
            set_error("term %d: CSR must be %d x %d with rowptr, col and val_re", i, n, n);
            return NEP_ERR_ARG;
        }
        if (c.rowptr[0] != 0) { set_error("term %d: rowptr[0] must be 0", i); return NEP_ERR_ARG; }
        for (int r = 0; r < n; ++r) {
            if (c.rowptr[r + 1] < c.rowptr[r]) { set_error("term %d: rowptr decreases at row %d", i, r); return NEP_ERR_ARG; }
            for (int64_t e = c.rowptr[r]; e < c.rowptr[r + 1]; ++e) {
                if (c.col[e] < 0 || c.col[e] >= n) { set_error("term %d: column index out of range in row %d", i, r); return NEP_ERR_ARG; }
                if (e > c.rowptr[r] && c.col[e] <= c.col[e - 1]) {
                    set_error("term %d: column indices of row %d not strictly increasing", i, r);
                    return NEP_ERR_ARG;
                }
            }
        }
    }
    nep_split* h = new nep_split();
    h->n = n;
    h->nterms = nterms;
    // union pattern: merge the sorted column lists row by row
    h->rowptr.assign(n + 1, 0);
    std::vector<int32_t> buf;
    for (int r = 0; r < n; ++r) {
        buf.clear();
        for (int i = 0; i < nterms; ++i)
            for (int64_t e = A[i].rowptr[r]; e < A[i].rowptr[r + 1]; ++e) buf.push_back(A[i].col[e]);
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        h->col.insert(h->col.end(), buf.begin(), buf.end());
        h->rowptr[r + 1] = (int64_t)h->col.size();
    }
    h->nnz = (int64_t)h->col.size();
    h->val.assign((size_t)nterms * h->nnz, 0.0);
    h->val_im.assign((size_t)nterms * h->nnz, 0.0);
    h->norms.assign(nterms, 0.0);
    for (int i = 0; i < nterms; ++i) {
        double nrm = 0.0;
        for (int r = 0; r < n; ++r) {
            int64_t u = h->rowptr[r];
            double rs = 0.0;
            for (int64_t e = A[i].rowptr[r]; e < A[i].rowptr[r + 1]; ++e) {
                while (h->col[u] != A[i].col[e]) ++u;
                const double re = A[i].val_re[e], im = A[i].val_im ? A[i].val_im[e] : 0.0;
                h->val[(size_t)i * h->nnz + u] = re;
                h->val_im[(size_t)i * h->nnz + u] = im;
                if (im != 0.0) h->complex_vals = true;
                rs += std::hypot(re, im);
            }
            nrm = std::max(nrm, rs);
        }
        h->norms[i] = nrm;
    }
    // column view of the union pattern (counting sort by column, rows ascending) and ||A_i||_1
    h->colptr.assign(n + 1, 0);
    for (int64_t e = 0; e < h->nnz; ++e) ++h->colptr[h->col[e] + 1];
    for (int c = 0; c < n; ++c) h->colptr[c + 1] += h->colptr[c];
    h->cidx.assign(h->nnz, 0);
    h->crow.assign(h->nnz, 0);
    {
        std::vector<int64_t> fill(h->colptr.begin(), h->colptr.end() - 1);
        for (int r = 0; r < n; ++r)
            for (int64_t e = h->rowptr[r]; e < h->rowptr[r + 1]; ++e) {
                const int64_t k = fill[h->col[e]]++;
                h->cidx[k] = e;
                h->crow[k] = r;
            }
    }
    h->norms1.assign(nterms, 0.0);
    for (int i = 0; i < nterms; ++i)
        for (int c = 0; c < n; ++c) {
            double cs = 0.0;
            for (int64_t k = h->colptr[c]; k < h->colptr[c + 1]; ++k) {
                const size_t e = (size_t)i * h->nnz + h->cidx[k];
                cs += std::hypot(h->val[e], h->val_im[e]);
            }
            h->norms1[i] = std::max(h->norms1[i], cs);
        }
    for (int r = 0; r < n; ++r)
        for (int64_t e = h->rowptr[r]; e < h->rowptr[r + 1]; ++e) {
            h->kl = std::max(h->kl, r - h->col[e]);
            h->ku = std::max(h->ku, h->col[e] - r);
        }
    h->ldab = 2 * h->kl + h->ku + 1;
    h->ext.resize(nterms);
    for (int i = 0; i < nterms; ++i) {
        const int root = flatten_fn(h, &f[i], 0);
        if (root < 0) { delete h; return NEP_ERR_ARG; }
        h->roots.push_back(root);
        if (f[i].kind == NEP_FN_CALLBACK || f[i].kind == NEP_FN_TABLE) {
            ExtTerm& e = h->ext[i];
            e.kind = f[i].kind;
            e.eval = f[i].eval;
            e.ctx = f[i].ctx;
            if (e.kind == NEP_FN_CALLBACK && !e.eval) { set_error("term %d: NEP_FN_CALLBACK needs eval", i); delete h; return NEP_ERR_ARG; }
            if (e.kind == NEP_FN_TABLE) {
                if (!f[i].table || f[i].table_count < 1) { set_error("term %d: NEP_FN_TABLE needs table and table_count >= 1", i); delete h; return NEP_ERR_ARG; }
                for (int k = 0; k < f[i].table_count; ++k) e.table.push_back(mk(f[i].table[2 * k], f[i].table[2 * k + 1]));
            }
            h->has_ext = true;
        }
    }
    cudaGetDevice(&h->device);
    int rc = NEP_OK;
    if ((rc = upload(&h->d_rowptr, h->rowptr)) || (rc = upload(&h->d_col, h->col)) || (rc = upload(&h->d_val, h->val)) ||
        (rc = upload(&h->d_val_im, h->val_im)) || (rc = upload(&h->d_norms, h->norms)) ||
        (rc = upload(&h->d_norms1, h->norms1)) || (rc = upload(&h->d_colptr, h->colptr)) ||
        (rc = upload(&h->d_cidx, h->cidx)) || (rc = upload(&h->d_crow, h->crow)) ||
        (rc = upload(&h->d_nodes, h->nodes)) || (rc = upload(&h->d_coef, h->coef)) || (rc = upload(&h->d_roots, h->roots)) ||
        (rc = cudaStreamSynchronize(0) == cudaSuccess ? NEP_OK : NEP_ERR_CUDA)) {
        free_split_device(h);
        delete h;
        return rc;
    }
    *out = h;
    return NEP_OK;
}

extern "C" int nep_destroy(nep_split_t h) {
    if (!h) return NEP_OK;
    free_split_device(h);
    delete h;
    return NEP_OK;
}

extern "C" int nep_split_info(nep_split_t h, int32_t* n, int32_t* nterms, int32_t* kl, int32_t* ku, int32_t* ldab) {
    if (!h) { set_error("null handle"); return NEP_ERR_ARG; }
    if (n) *n = h->n;
    if (nterms) *nterms = h->nterms;
    if (kl) *kl = h->kl;
    if (ku) *ku = h->ku;
    if (ldab) *ldab = h->ldab;
    return NEP_OK;
}

extern "C" void nep_opts_default(nep_opts* o) {
    if (!o) return;
    o->precision = NEP_PREC_MIXED;
    o->rank_tol = 1e-12;
    o->basis_tol = 1e-6;
    o->refine_tol = 1e-10;
    o->step_tol = 1e-14;
    o->refine_max = 10;
    o->eig_tol = 1e-8;
    o->newton_max = 30;
    o->newton_tol = 1e-14;
    o->seed = 0;
    o->symmetric = 0;
    o->newton_abandon = 8;
    o->refine_extrapolate = 1;
    o->lu_kernel = 0;
    o->solve_rh = 0;
}

extern "C" const char* nep_last_error(void) { return g_last_error.c_str(); }

extern "C" uint64_t nep_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" int nep_set_wait_limit(int64_t polls, int64_t* previous) {
    if (polls < 0) { set_error("nep_set_wait_limit: polls must be >= 0"); return NEP_ERR_ARG; }
    const long long old = g_wait_limit.exchange((long long)polls);
    if (previous) *previous = old;
    return NEP_OK;
}

// ============================================================================ region checks
typedef std::complex<double> C;

static bool in_closed_ellipse(C z, const nep_region* r) {
    const double x = (z.real() - r->center_re) / r->a, y = (z.imag() - r->center_im) / r->b;
    return x * x + y * y <= 1.0 + 1e-12;
}

// roots of a polynomial (highest degree first) by the Weierstrass (Durand-Kerner) iteration
static std::vector<C> poly_roots(const std::vector<C>& c) {
    std::vector<C> a(c.begin(), c.end());
    while (a.size() > 1 && std::abs(a[0]) == 0.0) a.erase(a.begin());
    const int d = (int)a.size() - 1;
    std::vector<C> z;
    if (d < 1) return z;
    for (auto& x : a) x /= a[0];
    double rad = 0;
    for (int i = 1; i <= d; ++i) rad = std::max(rad, std::pow(std::abs(a[i]), 1.0 / i));
    rad = 1.0 + 2.0 * rad;
    for (int i = 0; i < d; ++i) z.push_back(rad * std::polar(1.0, 0.4 + 2.0 * M_PI * i / d));
    for (int it = 0; it < 500; ++it) {
        double mx = 0;
        for (int i = 0; i < d; ++i) {
            C p = 1.0;
            for (int k = 1; k <= d; ++k) p = p * z[i] + a[k];
            C den = 1.0;
            for (int k = 0; k < d; ++k)
                if (k != i) den *= (z[i] - z[k]);
            const C dz = p / den;
            z[i] -= dz;
            mx = std::max(mx, std::abs(dz));
        }
        if (mx < 1e-15) break;
    }
    return z;
}

// Returns NEP_OK or NEP_ERR_REGION if a pole of a rational node or the cut of a sqrt node
// (argument alpha z) meets the closed ellipse. Nodes inside compositions are checked on
// their own argument only.
static int check_region_node(const nep_split* h, int k, const nep_region* r, bool top) {
    const FnNode& nd = h->nodes[k];
    const C alpha(nd.alpha.re, nd.alpha.im);
    if (nd.kind == NEP_FN_RATIONAL && nd.den_len > 1 && top) {
        std::vector<C> den;
        for (int t = 0; t < nd.den_len; ++t) den.push_back(C(h->coef[nd.den_off + t].re, h->coef[nd.den_off + t].im));
        for (const C& x : poly_roots(den)) {
            if (std::abs(alpha) == 0) continue;
            const C z = x / alpha;
            // a pole cancelled by the numerator is removable
            C p = 0;
            for (int t = 0; t < nd.num_len; ++t) p = p * x + C(h->coef[nd.num_off + t].re, h->coef[nd.num_off + t].im);
            if (std::abs(p) < 1e-12 * (1 + std::abs(x))) continue;
            if (in_closed_ellipse(z, r)) {
                set_error("pole of a rational term at (%g, %g) lies in the closed region", z.real(), z.imag());
                return NEP_ERR_REGION;
            }
        }
    } else if (nd.kind == NEP_FN_SQRT && top) {
        if (std::abs(alpha) == 0) return NEP_OK;
        // cut: alpha z - shift = -t, t >= 0  =>  z = (shift - t)/alpha; sample the ray densely
        const C s(nd.shift.re, nd.shift.im);
        const C z0 = s / alpha, d = -1.0 / alpha;
        const double span = 4.0 * (std::abs(C(r->center_re, r->center_im) - z0) + r->a + r->b) / std::abs(d);
        for (int i = 0; i <= 20000; ++i) {
            const double t = span * i / 20000.0;
            if (in_closed_ellipse(z0 + t * d, r)) {
                set_error("branch cut of a square-root term meets the closed region");
                return NEP_ERR_REGION;
            }
        }
    } else if (nd.kind == NEP_FN_COMBINE) {
        const bool inner_top = top && nd.op != NEP_OP_COMPOSE;
        nep_region rs = *r;
        // children see the argument alpha z: scale the region accordingly (circle/ellipse only
        // when alpha is real positive; otherwise checks apply to the outer argument only)
        if (!(nd.alpha.im == 0 && nd.alpha.re > 0)) return NEP_OK;
        rs.center_re *= nd.alpha.re;
        rs.center_im *= nd.alpha.re;
        rs.a *= nd.alpha.re;
        rs.b *= nd.alpha.re;
        int rc = check_region_node(h, nd.a, &rs, inner_top);
        if (rc) return rc;
        if (nd.op != NEP_OP_COMPOSE) return check_region_node(h, nd.b, &rs, inner_top);
        return check_region_node(h, nd.b, &rs, top);
    }
    return NEP_OK;
}

static int check_args(nep_split_t h, const nep_region* r, int N, int L, int M) {
    if (!h || !r) { set_error("null handle or region"); return NEP_ERR_ARG; }
    if (N < 2 || L < 1 || M < 1 || L > h->n) { set_error("need N >= 2, 1 <= L <= n, M >= 1"); return NEP_ERR_ARG; }
    if (!(r->a > 0) || !(r->b > 0)) { set_error("region semi-axes must be positive"); return NEP_ERR_ARG; }
    if ((int64_t)L * M > 512) { set_error("L*M = %d exceeds the supported 512", L * M); return NEP_ERR_UNSUPPORTED; }
    for (int i = 0; i < h->nterms; ++i) {
        const int rc = check_region_node(h, h->roots[i], r, true);
        if (rc) return rc;
    }
    return NEP_OK;
}

// ============================================================================ nodes / coefficients
static void make_nodes(const nep_region* r, int N, std::vector<zd>& z, std::vector<zd>& w, std::vector<zd>& zeta) {
    z.resize(N);
    w.resize(N);
    zeta.resize(N);
    for (int j = 0; j < N; ++j) {
        const double th = 2.0 * M_PI * (j + 0.5) / N;
        const double c = std::cos(th), s = std::sin(th);
        z[j] = mk(r->center_re + r->a * c, r->center_im + r->b * s);
        w[j] = mk(r->b * c / N, r->a * s / N);
        zeta[j] = mk(c, r->b * s / r->a);
    }
}

extern "C" int nep_nodes(const nep_region* r, int32_t N, double* z, double* w, double* zeta) {
    if (!r || N < 1) { set_error("nep_nodes: bad arguments"); return NEP_ERR_ARG; }
    std::vector<zd> zz, ww, qq;
    make_nodes(r, N, zz, ww, qq);
    if (z) memcpy(z, zz.data(), sizeof(zd) * N);
    if (w) memcpy(w, ww.data(), sizeof(zd) * N);
    if (zeta) memcpy(zeta, qq.data(), sizeof(zd) * N);
    return NEP_OK;
}

// f_i (and f_i' if dF) of every term at count points on the host, F[i + nterms k]: built-in terms by
// their function trees, host-supplied terms through the user's eval (one call per term for all
// points). A table term without eval has no values off its nodes: NEP_ERR_UNSUPPORTED.
int nep::host_terms(const nep_split* h, const zd* z, int count, zd* F, zd* dF) {
    std::vector<zd> f(count), df(count);
    for (int i = 0; i < h->nterms; ++i) {
        const ExtTerm& e = h->ext[i];
        if (e.kind < 0) {
            for (int k = 0; k < count; ++k) {
                const FnEval v = fn_eval(h->nodes.data(), h->coef.data(), h->roots[i], z[k]);
                F[i + (size_t)h->nterms * k] = v.f;
                if (dF) dF[i + (size_t)h->nterms * k] = v.df;
            }
            continue;
        }
        if (!e.eval) {
            set_error("term %d is tabulated at the quadrature nodes only: it needs eval for other points", i);
            return NEP_ERR_UNSUPPORTED;
        }
        if (count == 0) continue;
        e.eval(reinterpret_cast<const double*>(z), count, reinterpret_cast<double*>(f.data()),
               dF ? reinterpret_cast<double*>(df.data()) : nullptr, e.ctx);
        for (int k = 0; k < count; ++k) {
            F[i + (size_t)h->nterms * k] = f[k];
            if (dF) dF[i + (size_t)h->nterms * k] = df[k];
        }
    }
    return NEP_OK;
}

bool nep::split_has_host_terms(const nep_split* h) { return h && h->has_ext; }

extern "C" int nep_coefficients(nep_split_t h, int32_t N, const double* z, double* F, double* dF) {
    if (!h || !z || !F || N < 1) { set_error("nep_coefficients: bad arguments"); return NEP_ERR_ARG; }
    std::vector<zd> zz(N), FF((size_t)h->nterms * N), dd(dF ? (size_t)h->nterms * N : 0);
    for (int j = 0; j < N; ++j) zz[j] = mk(z[2 * j], z[2 * j + 1]);
    NEP_TRY(host_terms(h, zz.data(), N, FF.data(), dF ? dd.data() : nullptr));
    memcpy(F, FF.data(), sizeof(zd) * FF.size());
    if (dF) memcpy(dF, dd.data(), sizeof(zd) * dd.size());
    return NEP_OK;
}

// ============================================================================ tuning table
// Process-wide choices of nep_autotune (or a loaded cache file), keyed by the problem's shape: the plan
// of a matching shape takes them when its options leave lu_kernel / solve_rh at 0.
struct TuneKey {
    int n, kl, ku, L, precision;
    bool operator<(const TuneKey& o) const {
        return std::tie(n, kl, ku, L, precision) < std::tie(o.n, o.kl, o.ku, o.L, o.precision);
    }
};
struct TuneChoice {
    int lu_kernel = 0, solve_rh = 0;
    double ms = 0;
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneChoice> g_tune;

static bool tune_lookup(const TuneKey& k, TuneChoice* c) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(k);
    if (it == g_tune.end()) return false;
    *c = it->second;
    return true;
}

// ============================================================================ plan
struct nep_plan {
    nep_split_t h = nullptr;
    nep_region reg;
    nep_opts o;
    int N = 0, L = 0, M = 0, K = 0, LM = 0;
    int Np = 0;  // quadrature points solved: N, or N/2 under conjugate symmetry
    bool mixed = true;
    cudaStream_t alloc_stream = 0;
    // device buffers
    zd* F = nullptr;      // nterms x N
    zd* coef = nullptr;   // N x K (column k: w_j zeta_j^k)
    void* ab = nullptr;   // N x n x ldab of complex64/complex128
    void* ut = nullptr;   // N x n x (kl+ku+1): U by columns for the narrow-band sweeps (else unused)
    int* ipiv = nullptr;  // N x n
    int* info = nullptr;  // N
    double* tnorm = nullptr;
    zd* tval = nullptr;   // N x nnz
    zdf* tval_df = nullptr;  // N x nnz, complex64 plans: the double-float copy of tval
    zdf* V_df = nullptr;     // n x L, complex64 plans
    zd* V = nullptr;      // n x L
    zd* Y = nullptr;      // N x n x L
    zd* R = nullptr;      // N x n x L
    void* D = nullptr;    // N x n x L (solve precision)
    double* nrm = nullptr;  // N x L x 3
    double *dmax = nullptr, *ymax = nullptr, *prev = nullptr, *beta = nullptr;
    int *active = nullptr, *sweeps = nullptr, *nactive = nullptr;
    zd* S = nullptr;      // K x n x L
    zd* mu = nullptr;     // K x L x L
    zd* vpart = nullptr;  // chunks x K x L x L
    zd *H = nullptr, *Hs = nullptr, *Hw = nullptr, *U = nullptr, *W = nullptr;  // LM x LM
    double* sigma = nullptr;                                                     // LM
    zd *T1 = nullptr, *Bred = nullptr, *theta = nullptr, *Tv = nullptr, *Z = nullptr, *cand = nullptr;
    zd* XH = nullptr;     // n x LM
    zd *G = nullptr, *Gw = nullptr, *Wg = nullptr;
    double* lamg = nullptr;
    zd* Q = nullptr;      // n x LM
    zd* Y0 = nullptr;     // LM x LM
    zd* AQ = nullptr;     // nterms x n x LM
    zd* Bs = nullptr;     // nterms x LM x LM
    zd *lamn = nullptr, *Yn = nullptr, *Xc = nullptr, *Gx = nullptr;
    int *ok = nullptr, *its = nullptr, *order = nullptr, *scalars = nullptr, *eigstat = nullptr;
    double* eta = nullptr;
    zd* part = nullptr;
    size_t part_elems = 0;
    unsigned char* newton_scratch = nullptr;
    zf* bs32 = nullptr;  // complex64 copy of the projected B_i for Newton
    // host-supplied functions: Newton one step per launch with f_i, f_i' from the host
    double* nstate = nullptr;  // 4 per candidate: steps done, finished, FP64 phase, last |dlambda|
    zd* fvx = nullptr;         // per candidate: f_i then f_i' (2 nterms)
    void* eig_scratch = nullptr;
    JacobiWork jw{};
    int* h_pinned = nullptr;  // host-mapped scalars
    int lu_kernel = 0, solve_rh = 0;  // resolved tuning choices
    // last run
    int m = 0, kb = 0, max_sweeps_seen = 0, flags = 0, svd_sweeps = 0;
    double max_beta = 0;
    float ms[6] = {0, 0, 0, 0, 0, 0};
    cudaEvent_t ev[6] = {};
};

// Pinned host scalars of the plans, handed out from chunks that live as long as the process: a
// plan's cudaHostAlloc / cudaFreeHost pair would cost a pinning per plan and, at the free, a
// synchronisation of the whole device, stalling every other plan's stream (the request server
// creates and destroys a plan per request).
namespace nep {
static std::mutex g_pin_mu;
static std::vector<int*> g_pin_free;
int* pinned_slot_get() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr int kSlots = 64, kInts = 64;
        int* chunk = nullptr;
        if (cudaHostAlloc((void**)&chunk, sizeof(int) * kSlots * kInts, cudaHostAllocDefault) != cudaSuccess)
            return nullptr;
        for (int i = kSlots - 1; i >= 0; --i) g_pin_free.push_back(chunk + (size_t)kInts * i);
    }
    int* slot = g_pin_free.back();
    g_pin_free.pop_back();
    return slot;
}
void pinned_slot_put(int* slot) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(slot);
}
}  // namespace nep

static int plan_alloc(nep_plan* p) {
    const nep_split* h = p->h;
    const int n = h->n, N = p->Np, L = p->L, K = p->K, LM = p->LM, nt = h->nterms;
    cudaStream_t st = p->alloc_stream;
    const size_t esz = p->mixed ? sizeof(zf) : sizeof(zd);
    NEP_TRY(dalloc(&p->F, (size_t)nt * N, st));
    NEP_TRY(dalloc(&p->coef, (size_t)N * K, st));
    NEP_TRY(dalloc_raw(&p->ab, esz * (size_t)N * n * h->ldab, st));
    if (band_sweeps_fit(h->kl, h->ku)) NEP_TRY(dalloc_raw(&p->ut, esz * (size_t)N * n * (h->kl + h->ku + 1), st));
    NEP_TRY(dalloc(&p->ipiv, (size_t)N * n, st));
    NEP_TRY(dalloc(&p->info, N, st));
    NEP_TRY(dalloc(&p->tnorm, N, st));
    NEP_TRY(dalloc(&p->tval, (size_t)N * h->nnz, st));
    NEP_TRY(dalloc(&p->V, (size_t)n * L, st));
    NEP_TRY(dalloc(&p->Y, (size_t)N * n * L, st));
    if (p->mixed) {  // double-float refinement: no FP64 residual, split copies of T's values and V
        NEP_TRY(dalloc_raw(reinterpret_cast<void**>(&p->tval_df), sizeof(zdf) * (size_t)N * h->nnz, st));
        NEP_TRY(dalloc_raw(reinterpret_cast<void**>(&p->V_df), sizeof(zdf) * (size_t)n * L, st));
    } else {
        NEP_TRY(dalloc(&p->R, (size_t)N * n * L, st));
    }
    NEP_TRY(dalloc_raw(&p->D, esz * (size_t)N * n * L, st));
    NEP_TRY(dalloc(&p->nrm, (size_t)N * L * 3, st));
    NEP_TRY(dalloc(&p->dmax, N, st));
    NEP_TRY(dalloc(&p->ymax, N, st));
    NEP_TRY(dalloc(&p->prev, N, st));
    NEP_TRY(dalloc(&p->beta, N, st));
    NEP_TRY(dalloc(&p->active, N, st));
    NEP_TRY(dalloc(&p->sweeps, N, st));
    NEP_TRY(dalloc(&p->nactive, 1, st));
    NEP_TRY(dalloc(&p->S, (size_t)K * n * L, st));
    NEP_TRY(dalloc(&p->mu, (size_t)K * L * L, st));
    NEP_TRY(dalloc(&p->vpart, (size_t)ceil_div(n, 128) * K * L * L, st));
    const size_t lm2 = (size_t)LM * LM;
    NEP_TRY(dalloc(&p->H, lm2, st));
    NEP_TRY(dalloc(&p->Hs, lm2, st));
    NEP_TRY(dalloc(&p->Hw, lm2, st));
    NEP_TRY(dalloc(&p->U, lm2, st));
    NEP_TRY(dalloc(&p->W, lm2, st));
    NEP_TRY(dalloc(&p->sigma, LM, st));
    NEP_TRY(dalloc(&p->T1, lm2, st));
    NEP_TRY(dalloc(&p->Bred, lm2, st));
    NEP_TRY(dalloc(&p->theta, LM, st));
    NEP_TRY(dalloc(&p->Tv, lm2, st));
    NEP_TRY(dalloc(&p->Z, lm2, st));
    NEP_TRY(dalloc(&p->cand, LM, st));
    NEP_TRY(dalloc(&p->XH, (size_t)n * LM, st));
    NEP_TRY(dalloc(&p->G, lm2, st));
    NEP_TRY(dalloc(&p->Gw, lm2, st));
    NEP_TRY(dalloc(&p->Wg, lm2, st));
    NEP_TRY(dalloc(&p->lamg, LM, st));
    NEP_TRY(dalloc(&p->Q, (size_t)n * LM, st));
    NEP_TRY(dalloc(&p->Y0, lm2, st));
    NEP_TRY(dalloc(&p->AQ, (size_t)nt * n * LM, st));
    NEP_TRY(dalloc(&p->Bs, (size_t)nt * lm2, st));
    NEP_TRY(dalloc(&p->lamn, LM, st));
    NEP_TRY(dalloc(&p->Yn, lm2, st));
    NEP_TRY(dalloc(&p->Xc, (size_t)n * LM, st));
    NEP_TRY(dalloc(&p->Gx, lm2, st));
    NEP_TRY(dalloc(&p->ok, LM, st));
    NEP_TRY(dalloc(&p->its, LM, st));
    NEP_TRY(dalloc(&p->order, LM + 1, st));
    NEP_TRY(dalloc(&p->scalars, 8, st));
    NEP_TRY(dalloc(&p->eigstat, 1, st));
    NEP_TRY(dalloc(&p->eta, LM, st));
    p->part_elems = std::max<size_t>(16 * lm2, 1 << 16);
    NEP_TRY(dalloc(&p->part, p->part_elems, st));
    NEP_TRY(dalloc_raw((void**)&p->bs32, sizeof(zf) * (size_t)nt * LM * LM, st));
    if (newton_scratch_bytes(LM, nt) > 200 * 1024 || h->has_ext)
        NEP_TRY(dalloc_raw((void**)&p->newton_scratch, (size_t)LM * newton_scratch_bytes(LM, nt), st));
    if (h->has_ext) {
        NEP_TRY(dalloc(&p->nstate, (size_t)4 * LM, st));
        NEP_TRY(dalloc(&p->fvx, (size_t)2 * nt * LM, st));
    }
    NEP_TRY(dalloc_raw(&p->eig_scratch, sizeof(zf) * (size_t)LM * ((size_t)LM * (LM + 1) + 2 * LM) + 256, st));
    NEP_TRY(dalloc(&p->jw.Vm, lm2, st));
    NEP_TRY(dalloc(&p->jw.flags, 2, st));
    NEP_TRY(dalloc(&p->jw.sweeps, 1, st));
    NEP_TRY(dalloc(&p->jw.bar, 2, st));
    NEP_TRY(dalloc(&p->jw.err, 1, st));
    if (g_dry) return NEP_OK;
    NEP_CUDA(cudaMemsetAsync(p->jw.err, 0, sizeof(int), st));
    p->h_pinned = pinned_slot_get();
    if (!p->h_pinned) { set_error("no pinned host memory for the plan's scalars"); return NEP_ERR_NOMEM; }
    for (auto& e : p->ev) NEP_CUDA(cudaEventCreate(&e));
    return NEP_OK;
}

static void plan_free(nep_plan* p) {
    cudaStream_t st = p->alloc_stream;
    void* bufs[] = {p->F, p->coef, p->ab, p->ut, p->ipiv, p->info, p->tnorm, p->tval, p->tval_df, p->V_df, p->V, p->Y, p->R, p->D, p->nrm,
                    p->dmax, p->ymax, p->prev, p->beta, p->active, p->sweeps, p->nactive, p->S, p->mu, p->vpart,
                    p->H, p->Hs, p->Hw, p->U, p->W, p->sigma, p->T1, p->Bred, p->theta, p->Tv, p->Z, p->cand,
                    p->XH, p->G, p->Gw, p->Wg, p->lamg, p->Q, p->Y0, p->AQ, p->Bs, p->lamn, p->Yn, p->Xc, p->Gx,
                    p->ok, p->its, p->order, p->scalars, p->eigstat, p->eta, p->part, p->newton_scratch, p->bs32,
                    p->eig_scratch, p->jw.Vm, p->jw.flags, p->jw.sweeps, p->jw.bar, p->jw.err};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, st);
    cudaStreamSynchronize(st);
    if (p->h_pinned) pinned_slot_put(p->h_pinned);
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
}

namespace nep {
// Device bytes a plan for (h, N, L, M, precision) allocates (the same list as plan_alloc).
size_t plan_footprint(nep_split_t h, int N, int L, int M, int precision, int symmetric) {
    nep_plan p;
    p.h = h;
    p.N = N;
    p.Np = symmetric ? N / 2 : N;
    p.L = L;
    p.M = M;
    p.K = 2 * M;
    p.LM = L * M;
    p.mixed = precision == NEP_PREC_MIXED;
    g_dry = true;
    g_dry_bytes = 0;
    plan_alloc(&p);
    g_dry = false;
    return g_dry_bytes;
}
int plan_create_internal(nep_split_t h, const nep_region* r, int32_t N, int32_t L, int32_t M, const nep_opts* o,
                         cudaStream_t alloc_stream, nep_plan_t* out);
}  // namespace nep

extern "C" int nep_plan_create(nep_split_t h, const nep_region* r, int32_t N, int32_t L, int32_t M, const nep_opts* o,
                               nep_plan_t* out) {
    return plan_create_internal(h, r, N, L, M, o, 0, out);
}

int nep::plan_create_internal(nep_split_t h, const nep_region* r, int32_t N, int32_t L, int32_t M, const nep_opts* o,
                              cudaStream_t alloc_stream, nep_plan_t* out) {
    if (!out) { set_error("out is NULL"); return NEP_ERR_ARG; }
    *out = nullptr;
    NEP_TRY(check_args(h, r, N, L, M));
    configure_pool_once();
    nep_plan* p = new nep_plan();
    p->alloc_stream = alloc_stream;
    p->h = h;
    p->reg = *r;
    if (o) p->o = *o;
    else nep_opts_default(&p->o);
    if (p->o.precision != NEP_PREC_FP64 && p->o.precision != NEP_PREC_MIXED) {
        delete p;
        set_error("precision must be NEP_PREC_FP64 or NEP_PREC_MIXED");
        return NEP_ERR_ARG;
    }
    p->N = N;
    p->L = L;
    p->M = M;
    p->K = 2 * M;
    p->LM = L * M;
    p->mixed = p->o.precision == NEP_PREC_MIXED;
    {
        TuneChoice tc;
        const bool tuned = tune_lookup(TuneKey{h->n, h->kl, h->ku, L, p->o.precision}, &tc);
        p->lu_kernel = p->o.lu_kernel ? p->o.lu_kernel : (tuned ? tc.lu_kernel : 0);
        p->solve_rh = p->o.solve_rh ? p->o.solve_rh : (tuned ? tc.solve_rh : 0);
        if (p->lu_kernel < 0 || p->lu_kernel > 3 || !(p->solve_rh == 0 || p->solve_rh == 1 || p->solve_rh == 2 ||
                                                     p->solve_rh == 4)) {
            delete p;
            set_error("lu_kernel must be 0..3 and solve_rh 0, 1, 2 or 4");
            return NEP_ERR_ARG;
        }
    }
    p->Np = N;
    for (int i = 0; i < h->nterms; ++i) {
        const ExtTerm& e = h->ext[i];
        if (e.kind == NEP_FN_TABLE && (int)e.table.size() != N) {
            delete p;
            set_error("term %d is tabulated at %d nodes, the solve has N = %d", i, (int)e.table.size(), N);
            return NEP_ERR_ARG;
        }
        if (e.kind == NEP_FN_TABLE && !e.eval) {
            delete p;
            set_error("term %d is tabulated at the nodes only: the extraction step needs its values elsewhere "
                      "(give eval, or use the assembly and solve entry points with the table)", i);
            return NEP_ERR_UNSUPPORTED;
        }
    }
    std::vector<zd> z, w, zeta;
    make_nodes(r, N, z, w, zeta);
    if (p->o.symmetric) {
        // conjugate symmetry: z_{N-1-j} = conj z_j needs a real centre and an even N; T(conj z) =
        // conj T(z) needs real A_i and f_i(conj z) = conj f_i(z) (checked on the nodes)
        std::string why;
        if (N % 2) why = "N is odd";
        else if (r->center_im != 0.0) why = "the region's centre is not real";
        else if (h->complex_vals) {
            for (double v : h->val_im)
                if (v != 0.0) { why = "some A_i has complex entries"; break; }
        }
        for (int j = 0; j < N / 2 && why.empty(); ++j)
            for (int i = 0; i < h->nterms; ++i) {
                zd f, g;
                const ExtTerm& e = h->ext[i];
                if (e.kind == NEP_FN_TABLE) {  // conj z_j is the node N-1-j
                    f = e.table[j];
                    g = e.table[N - 1 - j];
                } else if (e.kind == NEP_FN_CALLBACK) {
                    const zd zz[2] = {z[j], conj(z[j])};
                    zd ff[2];
                    e.eval(reinterpret_cast<const double*>(zz), 2, reinterpret_cast<double*>(ff), nullptr, e.ctx);
                    f = ff[0];
                    g = ff[1];
                } else {
                    f = fn_eval(h->nodes.data(), h->coef.data(), h->roots[i], z[j]).f;
                    g = fn_eval(h->nodes.data(), h->coef.data(), h->roots[i], conj(z[j])).f;
                }
                const double d = std::hypot(g.re - f.re, g.im + f.im), a = std::hypot(f.re, f.im);
                if (!(d <= 1e-13 * std::max(a, 1e-300))) { why = "some f_i is not real (f(conj z) != conj f(z))"; break; }
            }
        if (!why.empty()) {
            delete p;
            set_error("symmetric quadrature not applicable: %s", why.c_str());
            return NEP_ERR_ARG;
        }
        p->Np = N / 2;  // nodes j < N/2 have Im z > 0; node N-1-j is their conjugate
    }
    int rc = plan_alloc(p);
    if (rc) {
        plan_free(p);
        delete p;
        return rc;
    }
    // coefficient table and moment weights of the solved nodes (host, FP64) -> device
    const int Np = p->Np;
    std::vector<zd> F((size_t)h->nterms * Np), coef((size_t)Np * p->K);
    if (h->has_ext) {
        // tabulated terms from their tables, callbacks through eval (one call per term), built-in
        // terms by their function trees
        for (int i = 0; i < h->nterms; ++i) {
            const ExtTerm& e = h->ext[i];
            if (e.kind == NEP_FN_TABLE) {
                for (int j = 0; j < Np; ++j) F[i + (size_t)h->nterms * j] = e.table[j];
            } else if (e.kind == NEP_FN_CALLBACK) {
                std::vector<zd> ff(Np);
                e.eval(reinterpret_cast<const double*>(z.data()), Np, reinterpret_cast<double*>(ff.data()), nullptr, e.ctx);
                for (int j = 0; j < Np; ++j) F[i + (size_t)h->nterms * j] = ff[j];
            } else {
                for (int j = 0; j < Np; ++j) F[i + (size_t)h->nterms * j] = fn_eval(h->nodes.data(), h->coef.data(), h->roots[i], z[j]).f;
            }
        }
    }
    for (int j = 0; j < Np; ++j) {
        if (!h->has_ext)
            for (int i = 0; i < h->nterms; ++i) F[i + (size_t)h->nterms * j] = fn_eval(h->nodes.data(), h->coef.data(), h->roots[i], z[j]).f;
        zd pw = mk(1.0, 0.0);
        for (int k = 0; k < p->K; ++k) {
            coef[j + (size_t)Np * k] = w[j] * pw;
            pw = pw * zeta[j];
        }
    }
    if (cudaMemcpyAsync(p->F, F.data(), sizeof(zd) * F.size(), cudaMemcpyHostToDevice, p->alloc_stream) != cudaSuccess ||
        cudaMemcpyAsync(p->coef, coef.data(), sizeof(zd) * coef.size(), cudaMemcpyHostToDevice, p->alloc_stream) != cudaSuccess ||
        cudaStreamSynchronize(p->alloc_stream) != cudaSuccess) {
        set_error("upload of the coefficient tables failed");
        plan_free(p);
        delete p;
        return NEP_ERR_CUDA;
    }
    *out = p;
    return NEP_OK;
}

extern "C" int nep_plan_destroy(nep_plan_t p) {
    if (!p) return NEP_OK;
    plan_free(p);
    delete p;
    return NEP_OK;
}

template <typename T>
static int run_solves(nep_plan* p, cudaStream_t st) {
    const SplitDev s = p->h->dev();
    const int N = p->Np, n = s.n, L = p->L;
    cx<T>* ab = reinterpret_cast<cx<T>*>(p->ab);
    cx<T>* D = reinterpret_cast<cx<T>*>(p->D);
    NEP_CUDA(cudaEventRecord(p->ev[0], st));
    NEP_TRY(launch_assemble<T>(s, N, p->F, ab, p->tnorm, p->tval, st));
    NEP_CUDA(cudaEventRecord(p->ev[1], st));
    NEP_TRY(launch_band_lu<T>(s, N, ab, p->ipiv, p->info, nullptr, st, p->lu_kernel));
    cx<T>* ut = reinterpret_cast<cx<T>*>(p->ut);
    if (ut) NEP_TRY(band_transpose_u<T>(s, N, ab, ut, st));
    NEP_CUDA(cudaEventRecord(p->ev[2], st));
    constexpr bool df = sizeof(T) == 4;  // complex64 factors: double-float refinement
    zdf* Ydf = reinterpret_cast<zdf*>(p->Y);
    NEP_TRY(launch_convert_rhs<T>(N, n, L, p->V, D, st));
    NEP_TRY(launch_band_solve<T>(s, N, ab, ut, p->ipiv, L, D, nullptr, st, p->solve_rh));
    if constexpr (df) {
        NEP_TRY(launch_split_df((int64_t)N * s.nnz, p->tval, p->tval_df, st));
        NEP_TRY(launch_split_df((int64_t)n * L, p->V, p->V_df, st));
        NEP_TRY(launch_widen_df(N, n, L, D, Ydf, st));
    } else {
        NEP_TRY(launch_widen<T>(N, n, L, D, p->Y, st));
    }
    NEP_TRY(launch_fill_int(N, p->active, 1, st));
    NEP_CUDA(cudaMemsetAsync(p->prev, 0, sizeof(double) * N, st));
    NEP_CUDA(cudaMemsetAsync(p->sweeps, 0, sizeof(int) * N, st));
    NEP_TRY(launch_drop_singular(N, n, L, p->info, p->Y, p->active, p->beta, st));  // zero bytes either way
    for (int sweep = 0; sweep < p->o.refine_max; ++sweep) {
        if constexpr (df) {
            NEP_TRY(launch_split_residual_df(s, N, p->tval_df, L, p->V_df, Ydf, D, p->nrm, p->active, st));
        } else {
            NEP_TRY(launch_split_residual(s, N, p->tval, L, p->V, p->Y, p->R, p->nrm, p->active, st));
            NEP_TRY(launch_refine_prepare<T>(N, n, L, p->R, D, p->active, st));
        }
        NEP_TRY(launch_band_solve<T>(s, N, ab, ut, p->ipiv, L, D, p->active, st, p->solve_rh));
        if constexpr (df) NEP_TRY(launch_refine_update_df(N, n, L, D, Ydf, p->dmax, p->ymax, p->active, st));
        else NEP_TRY(launch_refine_update<T>(N, n, L, D, p->Y, p->dmax, p->ymax, p->active, st));
        NEP_TRY(launch_refine_decide(N, L, sweep, p->o.refine_max, p->o.refine_tol, p->o.step_tol, p->o.refine_extrapolate, p->nrm, p->tnorm,
                                     p->dmax, p->ymax, p->prev, p->beta, p->active, p->sweeps, p->nactive, st));
        NEP_CUDA(cudaMemcpyAsync(p->h_pinned, p->nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
        NEP_CUDA(cudaStreamSynchronize(st));
        if (p->h_pinned[0] == 0) break;
    }
    NEP_CUDA(cudaEventRecord(p->ev[3], st));  // complex64 factors: Y stays double-float for the moments
    return NEP_OK;
}

// f_i (and f_i' when with_d) at the m device values lam_dev, evaluated on the host (host-supplied
// functions) into p->fvx: per candidate f_i then f_i'. Only finite values are handed to the
// functions; a candidate with a non-finite value gets zeros (its eta is then infinite).
static int host_values_at(nep_plan* p, const zd* lam_dev, int m, bool with_d, cudaStream_t st,
                          const std::vector<char>* skip = nullptr) {
    const int nt = p->h->nterms;
    std::vector<zd> lam(m), fv((size_t)2 * nt * m, mk(0.0, 0.0));
    NEP_CUDA(cudaMemcpyAsync(lam.data(), lam_dev, sizeof(zd) * m, cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    std::vector<int> idx;
    std::vector<zd> zs;
    for (int c = 0; c < m; ++c)
        if (std::isfinite(lam[c].re) && std::isfinite(lam[c].im) && !(skip && (*skip)[c])) {
            idx.push_back(c);
            zs.push_back(lam[c]);
        }
    const int cnt = (int)idx.size();
    std::vector<zd> F((size_t)nt * cnt), dF(with_d ? (size_t)nt * cnt : 0);
    NEP_TRY(host_terms(p->h, zs.data(), cnt, F.data(), with_d ? dF.data() : nullptr));
    for (int q = 0; q < cnt; ++q)
        for (int i = 0; i < nt; ++i) {
            fv[(size_t)idx[q] * 2 * nt + i] = F[i + (size_t)nt * q];
            if (with_d) fv[(size_t)idx[q] * 2 * nt + nt + i] = dF[i + (size_t)nt * q];
        }
    NEP_CUDA(cudaMemcpyAsync(p->fvx, fv.data(), sizeof(zd) * fv.size(), cudaMemcpyHostToDevice, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    return NEP_OK;
}

// Projected Newton for splits with host-supplied functions: one step per launch over all candidates,
// f_i and f_i' at each unfinished candidate's current iterate evaluated on the host in between (the
// same kernel, iterate kept in global memory; the same stopping rules).
static int newton_host_functions(nep_plan* p, const SplitDev& s, int kb, int m, double rad, cudaStream_t st) {
    NEP_CUDA(cudaMemsetAsync(p->nstate, 0, sizeof(double) * 4 * m, st));
    std::vector<double> stv((size_t)4 * m);
    std::vector<char> done(m, 0);
    for (int step = 1; step <= p->o.newton_max; ++step) {
        if (step > 1) {
            NEP_CUDA(cudaMemcpyAsync(stv.data(), p->nstate, sizeof(double) * 4 * m, cudaMemcpyDeviceToHost, st));
            NEP_CUDA(cudaStreamSynchronize(st));
            bool any = false;
            for (int c = 0; c < m; ++c) {
                done[c] = stv[4 * (size_t)c + 1] != 0.0;
                any |= !done[c];
            }
            if (!any) break;
        }
        NEP_TRY(host_values_at(p, step == 1 ? p->cand : p->lamn, m, true, st, &done));
        NEP_TRY(launch_newton(s, kb, m, p->Bs, p->bs32, p->cand, p->Y0, kb, mk(p->reg.center_re, p->reg.center_im), rad,
                              p->reg.a, p->reg.b, p->o.newton_max, p->o.newton_abandon, p->o.newton_tol, p->lamn, p->Yn,
                              p->ok, p->its, p->newton_scratch, st, p->fvx, p->nstate, 1));
    }
    return NEP_OK;
}

// ----------------------------------------------------------------- several plans, shared launches
// The quadrature solves of several plans (problems of uneven n, bandwidth, N and L) with the banded
// LU and the substitution sweeps of all their points in shared launches: one per kernel instance
// (points of equal band shape class), the rest per plan. Each point runs the same kernel instance
// with the same arguments as in its plan alone, so every result is bitwise the plan's own.
template <typename T>
static int run_solves_batch(const std::vector<nep_plan*>& ps, cudaStream_t st) {
    StreamScratch scratch(st);
    std::vector<std::vector<PointDesc>> keep;  // host copies live until the launches that read them
    auto upload = [&](const std::vector<PointDesc>& v, PointDesc** out) -> int {
        keep.push_back(v);
        NEP_TRY(scratch.get(out, v.size()));
        NEP_CUDA(cudaMemcpyAsync(*out, keep.back().data(), sizeof(PointDesc) * v.size(), cudaMemcpyHostToDevice, st));
        return NEP_OK;
    };
    auto point = [&](nep_plan* p, int j, void* B, const int* active) {
        const nep_split* h = p->h;
        PointDesc d{};
        d.n = h->n, d.kl = h->kl, d.ku = h->ku, d.ldab = h->ldab, d.L = p->L;
        d.ab = reinterpret_cast<cx<T>*>(p->ab) + (int64_t)j * h->n * h->ldab;
        d.ut = p->ut ? reinterpret_cast<const cx<T>*>(p->ut) + (int64_t)j * h->n * (h->kl + h->ku + 1) : nullptr;
        d.ipiv = p->ipiv + (int64_t)j * h->n;
        d.info = p->info + j;
        d.B = B ? reinterpret_cast<cx<T>*>(B) + (int64_t)j * h->n * p->L : nullptr;
        d.active = active ? active + j : nullptr;
        return d;
    };
    // assembly, per plan
    for (nep_plan* p : ps) {
        const SplitDev s = p->h->dev();
        NEP_CUDA(cudaEventRecord(p->ev[0], st));
        NEP_TRY(launch_assemble<T>(s, p->Np, p->F, reinterpret_cast<cx<T>*>(p->ab), p->tnorm, p->tval, st));
        NEP_CUDA(cudaEventRecord(p->ev[1], st));
    }
    // LU: register-window instances and the tensor-core kernel over all points; other shapes per plan
    std::map<int, std::vector<PointDesc>> col;
    std::vector<PointDesc> tc[2];  // tensor-core LU with 3 and with 1 products
    for (nep_plan* p : ps) {
        const SplitDev s = p->h->dev();
        const bool tc_ok = sizeof(T) == 4 && p->lu_kernel != LU_SIMT && (p->lu_kernel != LU_AUTO || lu_tc_enabled()) &&
                           band_lu_tc_fits(s.kl);
        // the tensor-core kernel asked for by name on a narrow band (as launch_band_lu takes it)
        const bool tc_named = sizeof(T) == 4 && (p->lu_kernel == LU_TC3 || p->lu_kernel == LU_TC1) &&
                              band_lu_col_fits(s.kl, s.ku) && band_lu_tc_can(s.kl);
        if (tc_named) {
            for (int j = 0; j < p->Np; ++j) tc[p->lu_kernel == LU_TC1].push_back(point(p, j, nullptr, nullptr));
        } else if (band_lu_col_fits(s.kl, s.ku)) {
            for (int j = 0; j < p->Np; ++j) col[lu_col_instance(s.kl, s.ku)].push_back(point(p, j, nullptr, nullptr));
        } else if (tc_ok) {
            for (int j = 0; j < p->Np; ++j) tc[p->lu_kernel == LU_TC1].push_back(point(p, j, nullptr, nullptr));
        } else {
            NEP_TRY(launch_band_lu<T>(s, p->Np, reinterpret_cast<cx<T>*>(p->ab), p->ipiv, p->info, nullptr, st,
                                      p->lu_kernel));
        }
    }
    for (auto& g : col) {
        PointDesc* pd = nullptr;
        NEP_TRY(upload(g.second, &pd));
        NEP_TRY(launch_band_lu_col_batch<T>(g.first, (int)g.second.size(), pd, st));
    }
    if (!tc[0].empty()) NEP_TRY(launch_band_lu_tc_batch(tc[0], st, 3));
    if (!tc[1].empty()) NEP_TRY(launch_band_lu_tc_batch(tc[1], st, 1));
    for (nep_plan* p : ps) {
        const SplitDev s = p->h->dev();
        if (p->ut) NEP_TRY(band_transpose_u<T>(s, p->Np, reinterpret_cast<cx<T>*>(p->ab), reinterpret_cast<cx<T>*>(p->ut), st));
        NEP_CUDA(cudaEventRecord(p->ev[2], st));
    }
    // one solve of every live plan's points: register-window sweeps in shared launches per shape key
    auto solve_all = [&](const std::vector<nep_plan*>& live, bool masked) -> int {
        std::map<std::tuple<int, int, int>, std::vector<PointDesc>> groups;
        std::map<std::tuple<int, int, int>, int> maxL;
        for (nep_plan* p : live) {
            const SplitDev s = p->h->dev();
            if (p->ut) {
                int a, b, r;
                sweep_key<T>(s.kl, s.ku, p->Np, p->L, &a, &b, &r, p->solve_rh);
                const auto key = std::make_tuple(a, b, r);
                for (int j = 0; j < p->Np; ++j) groups[key].push_back(point(p, j, p->D, masked ? p->active : nullptr));
                maxL[key] = std::max(maxL[key], p->L);
            } else {
                NEP_TRY(launch_band_solve<T>(s, p->Np, reinterpret_cast<cx<T>*>(p->ab), nullptr, p->ipiv, p->L,
                                             reinterpret_cast<cx<T>*>(p->D), masked ? p->active : nullptr, st,
                                             p->solve_rh));
            }
        }
        for (auto& g : groups) {
            PointDesc* pd = nullptr;
            NEP_TRY(upload(g.second, &pd));
            NEP_TRY(band_sweeps_batch<T>(std::get<0>(g.first), std::get<1>(g.first), std::get<2>(g.first),
                                         (int)g.second.size(), maxL[g.first], pd, st));
        }
        return NEP_OK;
    };
    for (nep_plan* p : ps) NEP_TRY(launch_convert_rhs<T>(p->Np, p->h->n, p->L, p->V, reinterpret_cast<cx<T>*>(p->D), st));
    NEP_TRY(solve_all(ps, false));
    constexpr bool df = sizeof(T) == 4;  // complex64 factors: double-float refinement, as run_solves
    for (nep_plan* p : ps) {
        const int N = p->Np, n = p->h->n, L = p->L;
        if constexpr (df) {
            NEP_TRY(launch_split_df((int64_t)N * p->h->nnz, p->tval, p->tval_df, st));
            NEP_TRY(launch_split_df((int64_t)n * L, p->V, p->V_df, st));
            NEP_TRY(launch_widen_df(N, n, L, reinterpret_cast<zf*>(p->D), reinterpret_cast<zdf*>(p->Y), st));
        } else {
            NEP_TRY(launch_widen<T>(N, n, L, reinterpret_cast<cx<T>*>(p->D), p->Y, st));
        }
        NEP_TRY(launch_fill_int(N, p->active, 1, st));
        NEP_CUDA(cudaMemsetAsync(p->prev, 0, sizeof(double) * N, st));
        NEP_CUDA(cudaMemsetAsync(p->sweeps, 0, sizeof(int) * N, st));
        NEP_TRY(launch_drop_singular(N, n, L, p->info, p->Y, p->active, p->beta, st));
    }
    // refinement: each plan's sweeps as alone, the solves of all live plans shared; one host read of
    // every plan's active count per sweep
    std::vector<nep_plan*> live;
    for (nep_plan* p : ps)
        if (p->o.refine_max > 0) live.push_back(p);
    for (int sweep = 0; !live.empty(); ++sweep) {
        for (nep_plan* p : live) {
            const SplitDev s = p->h->dev();
            if constexpr (df) {
                NEP_TRY(launch_split_residual_df(s, p->Np, p->tval_df, p->L, p->V_df, reinterpret_cast<zdf*>(p->Y),
                                                 reinterpret_cast<zf*>(p->D), p->nrm, p->active, st));
            } else {
                NEP_TRY(launch_split_residual(s, p->Np, p->tval, p->L, p->V, p->Y, p->R, p->nrm, p->active, st));
                NEP_TRY(launch_refine_prepare<T>(p->Np, s.n, p->L, p->R, reinterpret_cast<cx<T>*>(p->D), p->active, st));
            }
        }
        NEP_TRY(solve_all(live, true));
        for (nep_plan* p : live) {
            const SplitDev s = p->h->dev();
            if constexpr (df)
                NEP_TRY(launch_refine_update_df(p->Np, s.n, p->L, reinterpret_cast<zf*>(p->D),
                                                reinterpret_cast<zdf*>(p->Y), p->dmax, p->ymax, p->active, st));
            else
                NEP_TRY(launch_refine_update<T>(p->Np, s.n, p->L, reinterpret_cast<cx<T>*>(p->D), p->Y, p->dmax,
                                                p->ymax, p->active, st));
            NEP_TRY(launch_refine_decide(p->Np, p->L, sweep, p->o.refine_max, p->o.refine_tol, p->o.step_tol,
                                         p->o.refine_extrapolate, p->nrm, p->tnorm, p->dmax, p->ymax, p->prev, p->beta,
                                         p->active, p->sweeps, p->nactive, st));
            NEP_CUDA(cudaMemcpyAsync(p->h_pinned, p->nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
        }
        NEP_CUDA(cudaStreamSynchronize(st));
        std::vector<nep_plan*> next;
        for (nep_plan* p : live)
            if (p->h_pinned[0] != 0 && sweep + 1 < p->o.refine_max) next.push_back(p);
        live.swap(next);
    }
    for (nep_plan* p : ps) NEP_CUDA(cudaEventRecord(p->ev[3], st));
    return NEP_OK;
}

static int read_scalar(nep_plan* p, const int* dptr, int* out, cudaStream_t st) {
    NEP_CUDA(cudaMemcpyAsync(p->h_pinned, dptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    *out = p->h_pinned[0];
    return NEP_OK;
}

static int run_extract(nep_plan* p, cudaStream_t st) {
    const SplitDev s = p->h->dev();
    const int n = s.n, L = p->L, M = p->M, K = p->K, LM = p->LM, nt = s.nterms;
    // moments and Hankel matrices; under conjugate symmetry the nodes not solved contribute the
    // conjugates of the solved ones' terms: S_k = 2 Re sum_{Im z_j > 0} w_j zeta_j^k Y_j
    if (p->mixed) NEP_TRY(launch_moments_df(n, L, p->Np, K, p->coef, p->Y, p->S, st));  // Y back to FP64 too
    else NEP_TRY(launch_moments(n, L, p->Np, K, p->coef, p->Y, p->S, st));
    if (p->Np != p->N) NEP_TRY(launch_double_real(int64_t(K) * n * L, p->S, st));
    NEP_TRY(launch_vh_times(n, L, K, p->V, p->S, p->mu, p->vpart, st));
    NEP_TRY(launch_hankel_build(L, M, p->mu, p->H, p->Hs, st));
    NEP_CUDA(cudaEventRecord(p->ev[4], st));
    // SVD of H and numerical rank
    NEP_CUDA(cudaMemcpyAsync(p->Hw, p->H, sizeof(zd) * LM * LM, cudaMemcpyDeviceToDevice, st));
    // the QR preconditioner drops the trailing block of R once its Frobenius norm is below
    // 1e-14 |R_00| (and 1e-2 of the rank tolerance): singular values move by at most 1e-14
    // sigma_1, the size of the FP64 rounding error of a dense SVD of this order (n eps sigma_1),
    // and Jacobi runs only on the numerically nonzero part
    const double trunc = std::min(1e-14, 1e-2 * p->o.rank_tol);
    NEP_TRY(qrcp_jacobi_svd(LM, p->Hw, p->U, p->W, p->sigma, p->T1, p->Bred, p->Tv, p->theta, p->its, p->lamg,
                            p->scalars + 2, p->h_pinned + 8, trunc, p->jw, st));
    NEP_TRY(launch_rank(LM, p->sigma, p->o.rank_tol, p->scalars, st));
    int m = 0;
    NEP_TRY(read_scalar(p, p->scalars, &m, st));
    p->m = m;
    NEP_TRY(read_scalar(p, p->jw.sweeps, &p->svd_sweeps, st));
    p->kb = 0;
    if (m == 0) {
        NEP_CUDA(cudaMemsetAsync(p->order, 0, sizeof(int), st));
        return NEP_OK;
    }
    // reduced matrix U_m^H H< W_m Sigma_m^{-1} and its eigenpairs (FP32 Schur, seeds only)
    NEP_TRY(zgemm(LM, m, LM, 0, p->Hs, LM, p->W, LM, p->T1, LM, p->part, p->part_elems, st));
    NEP_TRY(zgemm(m, m, LM, 1, p->U, LM, p->T1, LM, p->Bred, m, p->part, p->part_elems, st));
    NEP_TRY(launch_scale_cols(m, m, p->Bred, m, p->sigma, 0, st));
    NEP_TRY(small_eig_fast<float>(m, p->Bred, p->theta, p->Tv, p->eigstat, p->eig_scratch, st));
    NEP_TRY(launch_candidates(m, p->theta, mk(p->reg.center_re, p->reg.center_im), p->reg.a, p->cand, st));
    // Hankel eigenvector estimates X_H = [S_0 .. S_{M-1}] W_m Sigma_m^{-1} T
    NEP_TRY(launch_scale_rows(m, m, p->Tv, m, p->sigma, st));
    NEP_TRY(zgemm(LM, m, m, 0, p->W, LM, p->Tv, m, p->Z, LM, p->part, p->part_elems, st));
    NEP_TRY(zgemm(n, m, LM, 0, p->S, n, p->Z, LM, p->XH, n, p->part, p->part_elems, st));
    NEP_TRY(launch_normalize_columns(n, m, p->XH, 0, nullptr, st));
    // orthonormal basis of the normalised columns: pivoted Cholesky of their Gram matrix
    NEP_TRY(zgemm(m, m, n, 1, p->XH, n, p->XH, n, p->G, m, p->part, p->part_elems, st));
    NEP_TRY(launch_pchol(m, p->G, p->o.basis_tol * p->o.basis_tol, p->scalars + 1, p->Wg, p->Gw, st));
    int kb = 0;
    NEP_TRY(read_scalar(p, p->scalars + 1, &kb, st));
    p->kb = kb;
    if (kb == 0) {
        NEP_CUDA(cudaMemsetAsync(p->order, 0, sizeof(int), st));
        return NEP_OK;
    }
    NEP_TRY(zgemm(n, kb, m, 0, p->XH, n, p->Wg, m, p->Q, n, p->part, p->part_elems, st));
    // Newton's starting vectors Q^H X_H = Z^H X_H^H X_H = Z^H G (Q = X_H Z): an m-sized product
    // in place of an n-sized one (they only seed the iteration)
    NEP_TRY(zgemm(kb, m, m, 1, p->Wg, m, p->G, m, p->Y0, kb, p->part, p->part_elems, st));
    // projected split form B_i = Q^H A_i Q, all terms in one product: the A_i Q blocks are
    // adjacent (n x nterms*kb) and so are the B_i (kb x nterms*kb)
    NEP_TRY(launch_term_spmm(s, kb, p->Q, p->AQ, st));
    NEP_TRY(zgemm(kb, nt * kb, n, 1, p->Q, n, p->AQ, n, p->Bs, kb, p->part, p->part_elems, st));
    // Newton from every Hankel candidate
    const double rad = 4.0 * std::max(p->reg.a, p->reg.b);
    if (p->h->has_ext) {
        NEP_TRY(newton_host_functions(p, s, kb, m, rad, st));
    } else {
        NEP_TRY(launch_newton(s, kb, m, p->Bs, p->bs32, p->cand, p->Y0, kb, mk(p->reg.center_re, p->reg.center_im), rad,
                              p->reg.a, p->reg.b, p->o.newton_max, p->o.newton_abandon, p->o.newton_tol, p->lamn, p->Yn,
                              p->ok, p->its, p->newton_scratch, st));
    }
    // eigenvectors, residuals, selection
    NEP_TRY(zgemm(n, m, kb, 0, p->Q, n, p->Yn, kb, p->Xc, n, p->part, p->part_elems, st));
    NEP_TRY(launch_normalize_columns(n, m, p->Xc, 1, nullptr, st));
    if (p->h->has_ext) {
        NEP_TRY(host_values_at(p, p->lamn, m, false, st));
        NEP_TRY(launch_eta(s, m, p->lamn, p->Xc, p->eta, st, p->fvx));
    } else {
        NEP_TRY(launch_eta(s, m, p->lamn, p->Xc, p->eta, st));
    }
    NEP_TRY(zgemm(m, m, n, 1, p->Xc, n, p->Xc, n, p->Gx, m, p->part, p->part_elems, st));
    NEP_TRY(launch_select(m, p->lamn, p->eta, p->ok, p->Gx, mk(p->reg.center_re, p->reg.center_im), p->reg.a, p->reg.b,
                          p->o.eig_tol, p->order, st));
    return NEP_OK;
}

extern "C" int nep_plan_execute(nep_plan_t p, const void* V_dev, void* stream) {
    if (!p || !V_dev) { set_error("nep_plan_execute: null plan or V"); return NEP_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->h->n, L = p->L;
    NEP_CUDA(cudaMemcpyAsync(p->V, V_dev, sizeof(zd) * (size_t)n * L, cudaMemcpyDeviceToDevice, st));
    if (p->Np != p->N) {
        // conjugate symmetry needs a real probe block
        NEP_TRY(launch_count_imag(int64_t(n) * L, p->V, p->scalars + 3, st));
        int nim = 0;
        NEP_TRY(read_scalar(p, p->scalars + 3, &nim, st));
        if (nim) { set_error("symmetric quadrature needs a real V (%d entries have an imaginary part)", nim); return NEP_ERR_ARG; }
    }
    NEP_CUDA(cudaMemsetAsync(p->jw.err, 0, sizeof(int), st));
    int rc = p->mixed ? run_solves<float>(p, st) : run_solves<double>(p, st);
    if (rc) return rc;
    NEP_TRY(run_extract(p, st));
    NEP_CUDA(cudaEventRecord(p->ev[5], st));
    int err = 0;
    NEP_TRY(read_scalar(p, p->jw.err, &err, st));
    if (err) { set_error("a bounded grid barrier of the Jacobi SVD timed out"); return NEP_ERR_INTERNAL; }
    return NEP_OK;
}

extern "C" int nep_plan_execute_batch(int32_t count, nep_plan_t* plans, const void* const* V_devs, void* stream) {
    if (count < 1 || !plans || !V_devs) { set_error("nep_plan_execute_batch: bad arguments"); return NEP_ERR_ARG; }
    std::vector<nep_plan*> ps;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !V_devs[i]) { set_error("nep_plan_execute_batch: null plan or V at %d", i); return NEP_ERR_ARG; }
        for (nep_plan* q : ps)
            if (q == plans[i]) { set_error("nep_plan_execute_batch: plan %d appears twice", i); return NEP_ERR_ARG; }
        if (plans[i]->mixed != plans[0]->mixed) { set_error("nep_plan_execute_batch: plans of one precision only"); return NEP_ERR_ARG; }
        if (plans[i]->h->has_ext) { set_error("nep_plan_execute_batch: callback or table terms are not batched"); return NEP_ERR_UNSUPPORTED; }
        ps.push_back(plans[i]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        nep_plan* p = ps[i];
        const int n = p->h->n, L = p->L;
        NEP_CUDA(cudaMemcpyAsync(p->V, V_devs[i], sizeof(zd) * (size_t)n * L, cudaMemcpyDeviceToDevice, st));
        if (p->Np != p->N) {
            NEP_TRY(launch_count_imag(int64_t(n) * L, p->V, p->scalars + 3, st));
            int nim = 0;
            NEP_TRY(read_scalar(p, p->scalars + 3, &nim, st));
            if (nim) { set_error("plan %d: symmetric quadrature needs a real V", i); return NEP_ERR_ARG; }
        }
        NEP_CUDA(cudaMemsetAsync(p->jw.err, 0, sizeof(int), st));
    }
    int rc = ps[0]->mixed ? run_solves_batch<float>(ps, st) : run_solves_batch<double>(ps, st);
    if (rc) return rc;
    for (nep_plan* p : ps) {
        NEP_TRY(run_extract(p, st));
        NEP_CUDA(cudaEventRecord(p->ev[5], st));
        int err = 0;
        NEP_TRY(read_scalar(p, p->jw.err, &err, st));
        if (err) { set_error("a bounded grid barrier of the Jacobi SVD timed out"); return NEP_ERR_INTERNAL; }
    }
    return NEP_OK;
}

// ----------------------------------------------------------------- autotuning
extern "C" int nep_tune_load(const char* path, int32_t* entries) {
    if (!path) { set_error("nep_tune_load: null path"); return NEP_ERR_ARG; }
    FILE* f = fopen(path, "r");
    if (!f) { set_error("nep_tune_load: cannot open %s", path); return NEP_ERR_ARG; }
    char line[512];
    int count = 0;
    while (fgets(line, sizeof line, f)) {
        TuneKey k{};
        TuneChoice c;
        if (sscanf(line, "nep-tune n=%d kl=%d ku=%d L=%d precision=%d lu_kernel=%d solve_rh=%d ms=%lf", &k.n, &k.kl,
                   &k.ku, &k.L, &k.precision, &c.lu_kernel, &c.solve_rh, &c.ms) == 8) {
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune[k] = c;  // later lines win
            ++count;
        }
    }
    fclose(f);
    if (entries) *entries = count;
    return NEP_OK;
}

extern "C" int nep_autotune(nep_split_t h, const nep_region* r, int32_t N, int32_t L, int32_t M, const nep_opts* o,
                            const void* V_dev, const char* cache_path, nep_tune_result* out, void* stream) {
    if (!h || !r || !V_dev || !out) { set_error("nep_autotune: bad arguments"); return NEP_ERR_ARG; }
    if (h->has_ext) { set_error("nep_autotune: callback or table terms are not tuned"); return NEP_ERR_UNSUPPORTED; }
    nep_opts base;
    if (o) base = *o;
    else nep_opts_default(&base);
    cudaStream_t st = (cudaStream_t)stream;
    const bool wide_c64 = base.precision == NEP_PREC_MIXED && h->kl > 64 && band_lu_tc_fits(h->kl);
    const std::vector<int> lus = wide_c64 ? std::vector<int>{LU_TC3, LU_TC1, LU_SIMT} : std::vector<int>{LU_AUTO};
    const std::vector<int> rhs = band_sweeps_fit(h->kl, h->ku) ? std::vector<int>{1, 2, 4} : std::vector<int>{0};
    *out = nep_tune_result{};
    double best = 1e300;
    cudaEvent_t e0, e1;
    NEP_CUDA(cudaEventCreate(&e0));
    NEP_CUDA(cudaEventCreate(&e1));
    int rc = NEP_OK;
    for (int lu : lus)
        for (int rh : rhs) {
            nep_opts oo = base;
            oo.lu_kernel = lu;
            oo.solve_rh = rh;
            nep_plan_t p = nullptr;
            if ((rc = nep_plan_create(h, r, N, L, M, &oo, &p))) break;
            // one pass to warm up, then the mean of two timed passes (device time, CUDA events)
            float ms = 0;
            rc = nep_plan_execute(p, V_dev, st);
            if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = NEP_ERR_CUDA;
            for (int it = 0; it < 2 && !rc; ++it) rc = nep_plan_execute(p, V_dev, st);
            if (!rc && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = NEP_ERR_CUDA;
            nep_result_t res = nullptr;
            if (!rc) rc = nep_plan_result(p, &res);
            nep_plan_destroy(p);
            if (rc) break;
            // accuracy gate: every quadrature solve at the backward-error target, no worse flags
            nep_result_info_t ri{};
            nep_result_info(res, &ri);
            const bool accurate = !(ri.flags & NEP_WARN_REFINE) && ri.max_backward <= base.refine_tol;
            nep_result_free(res);
            ++out->candidates;
            if (!accurate) continue;
            ++out->accurate;
            if (ms / 2 < best) {
                best = ms / 2;
                out->lu_kernel = lu;
                out->solve_rh = rh;
                out->ms = ms / 2;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (out->accurate == 0) { set_error("nep_autotune: no candidate met the accuracy target"); return NEP_ERR_INTERNAL; }
    const TuneKey k{h->n, h->kl, h->ku, L, base.precision};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[k] = TuneChoice{out->lu_kernel, out->solve_rh, out->ms};
    }
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (!f) { set_error("nep_autotune: cannot append to %s", cache_path); return NEP_ERR_ARG; }
        fprintf(f, "nep-tune n=%d kl=%d ku=%d L=%d precision=%d lu_kernel=%d solve_rh=%d ms=%.6f\n", k.n, k.kl, k.ku,
                k.L, k.precision, out->lu_kernel, out->solve_rh, out->ms);
        fclose(f);
    }
    return NEP_OK;
}

extern "C" int nep_plan_buffer(nep_plan_t p, const char* name, void** dev_ptr, size_t* bytes) {
    if (!p || !name || !dev_ptr) { set_error("nep_plan_buffer: bad arguments"); return NEP_ERR_ARG; }
    const nep_split* h = p->h;
    const size_t n = h->n, N = p->Np, L = p->L, K = p->K;
    const size_t esz = p->mixed ? sizeof(zf) : sizeof(zd);
    struct B { const char* nm; void* ptr; size_t bytes; } tab[] = {
        {"F", p->F, sizeof(zd) * h->nterms * N},   {"coef", p->coef, sizeof(zd) * N * K},
        {"ab", p->ab, esz * N * n * h->ldab},       {"ipiv", p->ipiv, sizeof(int) * N * n},
        {"ut", p->ut, p->ut ? esz * N * n * (h->kl + h->ku + 1) : 0},
        {"info", p->info, sizeof(int) * N},         {"Y", p->Y, sizeof(zd) * N * n * L},
        {"S", p->S, sizeof(zd) * K * n * L},        {"mu", p->mu, sizeof(zd) * K * L * L},
        {"sigma", p->sigma, sizeof(double) * p->LM}, {"tnorm", p->tnorm, sizeof(double) * N},
        {"beta", p->beta, sizeof(double) * N},      {"sweeps", p->sweeps, sizeof(int) * N},
        {"H", p->H, sizeof(zd) * p->LM * p->LM},
        {"newton_its", p->its, sizeof(int) * p->LM},  {"newton_ok", p->ok, sizeof(int) * p->LM},
        {"candidates", p->cand, sizeof(zd) * p->LM},  {"newton_lambda", p->lamn, sizeof(zd) * p->LM},
    };
    for (auto& b : tab)
        if (!strcmp(b.nm, name)) {
            *dev_ptr = b.ptr;
            if (bytes) *bytes = b.bytes;
            return NEP_OK;
        }
    set_error("unknown plan buffer '%s'", name);
    return NEP_ERR_ARG;
}

// ============================================================================ results
struct nep_result {
    int n = 0, nconv = 0, m = 0, flags = 0;
    std::vector<double> lam, X, resid, sigma;
    std::vector<int32_t> pt_sweeps, pt_info;  // per solved quadrature point
    std::vector<double> pt_beta;
    nep_result_info_t info{};
};

// ------------------------------------------------------------------ residual inverse iteration
extern "C" int nep_rii(nep_split_t h, int32_t precision, int32_t P, double* lam_dev, double* X_dev, double* eta_dev,
                       int32_t* its_dev, double tol, int32_t max_it, int32_t* iterations, void* stream) {
    if (h && h->has_ext) {
        set_error("this entry point evaluates the functions on the device: not available with callback or table terms");
        return NEP_ERR_UNSUPPORTED;
    }
    if (!h || P < 0 || max_it < 0 || (P > 0 && (!lam_dev || !X_dev || !eta_dev))) {
        set_error("nep_rii: bad arguments");
        return NEP_ERR_ARG;
    }
    if (precision != NEP_PREC_MIXED && precision != NEP_PREC_FP64) { set_error("nep_rii: bad precision"); return NEP_ERR_ARG; }
    if (iterations) *iterations = 0;
    if (P == 0) return NEP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const SplitDev s = h->dev();
    int* its = its_dev;
    if (!its) NEP_CUDA(cudaMallocAsync((void**)&its, sizeof(int) * (size_t)P, st));
    int k = 0;
    int rc = precision == NEP_PREC_MIXED
                 ? rii_polish<float>(s, P, (zd*)lam_dev, (zd*)X_dev, eta_dev, its, tol, max_it, &k, st)
                 : rii_polish<double>(s, P, (zd*)lam_dev, (zd*)X_dev, eta_dev, its, tol, max_it, &k, st);
    if (!its_dev) cudaFreeAsync(its, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NEP_ERR_CUDA;
    if (!rc && iterations) *iterations = k;
    return rc;
}

extern "C" int nep_plan_polish(nep_plan_t p, double tol, int32_t max_it, int32_t* polished, int32_t* iterations,
                               void* stream) {
    if (p && p->h && p->h->has_ext) {
        set_error("this entry point evaluates the functions on the device: not available with callback or table terms");
        return NEP_ERR_UNSUPPORTED;
    }
    if (!p || max_it < 0) { set_error("nep_plan_polish: bad arguments"); return NEP_ERR_ARG; }
    if (polished) *polished = 0;
    if (iterations) *iterations = 0;
    if (p->m <= 0 || p->kb <= 0) return NEP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->h->n, m = p->m;
    // the returned eigenpairs whose eta is not below tol
    std::vector<int> order(m + 1, 0);
    std::vector<double> eta(m);
    NEP_CUDA(cudaMemcpyAsync(order.data(), p->order, sizeof(int) * (m + 1), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaMemcpyAsync(eta.data(), p->eta, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    std::vector<int> idx;
    for (int q = 0; q < order[0]; ++q)
        if (!(eta[order[1 + q]] < tol)) idx.push_back(order[1 + q]);
    const int P = (int)idx.size();
    if (P == 0) return NEP_OK;
    int* didx = nullptr;
    zd *lam = nullptr, *X = nullptr;
    double* e = nullptr;
    int* its = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&didx, sizeof(int) * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&lam, sizeof(zd) * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&X, sizeof(zd) * (size_t)n * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&e, sizeof(double) * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&its, sizeof(int) * P, st));
    int rc = NEP_OK, k = 0;
    if (cudaMemcpyAsync(didx, idx.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = NEP_ERR_CUDA;
    if (!rc) rc = launch_rii_move(n, P, didx, p->lamn, p->Xc, p->eta, lam, X, e, 0, st);
    if (!rc) rc = p->mixed ? rii_polish<float>(p->h->dev(), P, lam, X, e, its, tol, max_it, &k, st)
                           : rii_polish<double>(p->h->dev(), P, lam, X, e, its, tol, max_it, &k, st);
    if (!rc) rc = launch_rii_move(n, P, didx, p->lamn, p->Xc, p->eta, lam, X, e, 1, st);
    for (void* b : {(void*)didx, (void*)lam, (void*)X, (void*)e, (void*)its}) cudaFreeAsync(b, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NEP_ERR_CUDA;
    if (!rc) {
        if (polished) *polished = P;
        if (iterations) *iterations = k;
    }
    return rc;
}

extern "C" int nep_left_eigvecs(nep_split_t h, int32_t precision, int32_t P, const double* lam_dev,
                                const double* X_dev, double* Y_dev, double* eta_dev, int32_t* its_dev, double tol,
                                int32_t max_it, int32_t* iterations, void* stream) {
    if (h && h->has_ext) {
        set_error("this entry point evaluates the functions on the device: not available with callback or table terms");
        return NEP_ERR_UNSUPPORTED;
    }
    if (!h || P < 0 || max_it < 1 || (P > 0 && (!lam_dev || !X_dev || !Y_dev || !eta_dev))) {
        set_error("nep_left_eigvecs: bad arguments");
        return NEP_ERR_ARG;
    }
    if (precision != NEP_PREC_MIXED && precision != NEP_PREC_FP64) {
        set_error("nep_left_eigvecs: bad precision");
        return NEP_ERR_ARG;
    }
    if (iterations) *iterations = 0;
    if (P == 0) return NEP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const SplitDev s = h->dev();
    int* its = its_dev;
    if (!its) NEP_CUDA(cudaMallocAsync((void**)&its, sizeof(int) * (size_t)P, st));
    int k = 0;
    int rc = precision == NEP_PREC_MIXED
                 ? left_eigvecs<float>(s, P, (const zd*)lam_dev, (const zd*)X_dev, (zd*)Y_dev, eta_dev, its, tol,
                                       max_it, &k, st)
                 : left_eigvecs<double>(s, P, (const zd*)lam_dev, (const zd*)X_dev, (zd*)Y_dev, eta_dev, its, tol,
                                        max_it, &k, st);
    if (!its_dev) cudaFreeAsync(its, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NEP_ERR_CUDA;
    if (!rc && iterations) *iterations = k;
    return rc;
}

extern "C" int nep_plan_left(nep_plan_t p, double tol, int32_t max_it, int32_t capacity, double* Y_dev,
                             double* eta_dev, int32_t* nconv, int32_t* iterations, void* stream) {
    if (p && p->h && p->h->has_ext) {
        set_error("this entry point evaluates the functions on the device: not available with callback or table terms");
        return NEP_ERR_UNSUPPORTED;
    }
    if (!p || max_it < 1 || capacity < 0 || (capacity > 0 && (!Y_dev || !eta_dev))) {
        set_error("nep_plan_left: bad arguments");
        return NEP_ERR_ARG;
    }
    if (nconv) *nconv = 0;
    if (iterations) *iterations = 0;
    if (p->m <= 0 || p->kb <= 0) return NEP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = p->h->n, m = p->m;
    std::vector<int> order(m + 1, 0);
    NEP_CUDA(cudaMemcpyAsync(order.data(), p->order, sizeof(int) * (m + 1), cudaMemcpyDeviceToHost, st));
    NEP_CUDA(cudaStreamSynchronize(st));
    const int P = order[0];
    if (nconv) *nconv = P;
    if (P == 0) return NEP_OK;
    if (P > capacity) {
        set_error("nep_plan_left: %d returned pairs, room for %d", P, capacity);
        return NEP_ERR_ARG;
    }
    int* didx = nullptr;
    zd *lam = nullptr, *X = nullptr;
    double* e = nullptr;
    int* its = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&didx, sizeof(int) * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&lam, sizeof(zd) * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&X, sizeof(zd) * (size_t)n * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&e, sizeof(double) * P, st));
    NEP_CUDA(cudaMallocAsync((void**)&its, sizeof(int) * P, st));
    int rc = NEP_OK, k = 0;
    // the returned pairs in the order of nep_plan_result
    if (cudaMemcpyAsync(didx, order.data() + 1, sizeof(int) * P, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = NEP_ERR_CUDA;
    if (!rc) rc = launch_rii_move(n, P, didx, p->lamn, p->Xc, p->eta, lam, X, e, 0, st);
    if (!rc) rc = p->mixed ? left_eigvecs<float>(p->h->dev(), P, lam, X, (zd*)Y_dev, eta_dev, its, tol, max_it, &k, st)
                           : left_eigvecs<double>(p->h->dev(), P, lam, X, (zd*)Y_dev, eta_dev, its, tol, max_it, &k, st);
    for (void* b : {(void*)didx, (void*)lam, (void*)X, (void*)e, (void*)its}) cudaFreeAsync(b, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NEP_ERR_CUDA;
    if (!rc && iterations) *iterations = k;
    return rc;
}

extern "C" int nep_apply_resolvent(int32_t n, int32_t P, const double* lam_dev, const double* X_dev,
                                   const double* Y_dev, int32_t nz, const double* z_dev, int32_t nv,
                                   const double* V_dev, double* out_dev, void* stream) {
    if (n < 1 || P < 0 || nz < 0 || nv < 0 || (P > 0 && (!lam_dev || !X_dev || !Y_dev)) ||
        (nz > 0 && nv > 0 && (!z_dev || !V_dev || !out_dev))) {
        set_error("nep_apply_resolvent: bad arguments");
        return NEP_ERR_ARG;
    }
    return apply_resolvent(n, P, (const zd*)lam_dev, (const zd*)X_dev, (const zd*)Y_dev, nz, (const zd*)z_dev, nv,
                           (const zd*)V_dev, (zd*)out_dev, (cudaStream_t)stream);
}

// ============================================================================ NLEIGS
struct NleigsParams {
    double tol;
    int dmax, nb, kmax, eig_ok;
    zd shift;
    uint64_t seed;
    double eig_tol;
    bool exact;
    bool toar;
    int max_restarts, keep, nev;
    double restart_tol;
};

// Krylov-Schur restart options of NLEIGS and Interpol on a cycle of kmax Arnoldi steps
static int ks_params(int max_restarts, int keep, double tol, int nev, int kmax, bool exact, KsOpts* ks) {
    if (max_restarts < 0 || max_restarts > 10000 || keep < 0 || tol < 0 || nev < 0) {
        set_error("restarts: need 0 <= max_restarts <= 10000, keep >= 0, restart_tol >= 0, nev >= 0");
        return NEP_ERR_ARG;
    }
    if (max_restarts > 0 && (kmax < 2 || keep >= kmax)) {
        set_error("restarts: need krylov >= 2 and keep < krylov (krylov %d, keep %d)", kmax, keep);
        return NEP_ERR_ARG;
    }
    ks->max_restarts = max_restarts;
    ks->keep = keep > 0 ? keep : std::max(1, kmax / 2);
    ks->tol = tol > 0 ? tol : (exact ? 1e-10 : 1e-6);
    ks->nev = nev;
    return NEP_OK;
}

static int nleigs_params(nep_split_t h, const nep_region* r, const nep_nleigs_opts* o, NleigsParams* q) {
    if (!h || !r) { set_error("null handle or region"); return NEP_ERR_ARG; }
    if (!(r->a > 0) || !(r->b > 0)) { set_error("region semi-axes must be positive"); return NEP_ERR_ARG; }
    nep_nleigs_opts z{};
    if (!o) o = &z;
    q->tol = o->tol > 0 ? o->tol : 1e-13;
    q->dmax = o->max_degree > 0 ? o->max_degree : 60;
    q->nb = o->nboundary > 0 ? o->nboundary : 1024;
    q->kmax = o->krylov > 0 ? o->krylov : 100;
    q->shift = o->has_shift ? mk(o->shift_re, o->shift_im) : mk(r->center_re, r->center_im);
    q->seed = o->seed;
    q->eig_tol = o->eig_tol > 0 ? o->eig_tol : 1e-8;
    q->exact = o->exact_solves != 0;
    q->toar = o->full_basis == 0;
    q->max_restarts = o->max_restarts;
    q->keep = o->keep;
    q->restart_tol = o->restart_tol;
    q->nev = o->nev;
    if (q->dmax > 63 || q->nb < 8 || q->nb > (1 << 20) || q->kmax > 512) {
        set_error("nleigs: max_degree <= 63, 8 <= nboundary <= 2^20, krylov <= 512");
        return NEP_ERR_ARG;
    }
    for (int i = 0; i < h->nterms; ++i) {
        const int rc = check_region_node(h, h->roots[i], r, true);
        if (rc) return rc;
    }
    return NEP_OK;
}

static int nleigs_interp_out(nep_split_t h, const nep_region* r, const nep_nleigs_opts* o, int32_t cap,
                             double* sigma, double* xi, double* beta, double* dd, int32_t* degree,
                             int32_t* converged, int32_t* nsing);

extern "C" int nep_nleigs_interpolation(nep_split_t h, const nep_region* r, const nep_nleigs_opts* o, int32_t cap,
                                        double* sigma, double* xi, double* beta, double* dd, int32_t* degree,
                                        int32_t* converged, int32_t* nsing) {
    if (h && h->has_ext) {
        set_error("this entry point evaluates the functions on the device: not available with callback or table terms");
        return NEP_ERR_UNSUPPORTED;
    }
    return nleigs_interp_out(h, r, o, cap, sigma, xi, beta, dd, degree, converged, nsing);
}

extern "C" int nep_nleigs_interpolation_fns(int32_t nterms, const nep_fn* f, const nep_region* r,
                                            const nep_nleigs_opts* o, int32_t cap, double* sigma, double* xi,
                                            double* beta, double* dd, int32_t* degree, int32_t* converged,
                                            int32_t* nsing) {
    if (nterms < 1 || nterms > 32 || !f) {
        set_error("nep_nleigs_interpolation_fns: need 1 <= nterms <= 32 and non-NULL f");
        return NEP_ERR_ARG;
    }
    // the function trees only, on the host: no matrices, no device memory
    nep_split h;
    h.nterms = nterms;
    for (int i = 0; i < nterms; ++i) {
        const int root = flatten_fn(&h, &f[i], 0);
        if (root < 0) return NEP_ERR_ARG;
        h.roots.push_back(root);
    }
    return nleigs_interp_out(&h, r, o, cap, sigma, xi, beta, dd, degree, converged, nsing);
}

static int nleigs_interp_out(nep_split_t h, const nep_region* r, const nep_nleigs_opts* o, int32_t cap,
                             double* sigma, double* xi, double* beta, double* dd, int32_t* degree,
                             int32_t* converged, int32_t* nsing) {
    NleigsParams q;
    NEP_TRY(nleigs_params(h, r, o, &q));
    NleigsInterp it;
    NEP_TRY(nleigs_interpolation(h->nodes, h->coef, h->roots, mk(r->center_re, r->center_im), r->a, r->b, q.tol,
                                 q.dmax, q.nb, &it));
    if (degree) *degree = it.d;
    if (converged) *converged = it.converged;
    if (nsing) *nsing = it.nsing;
    const int d1 = it.d + 1, nt = h->nterms;
    if ((sigma || xi || beta || dd) && cap < d1) {
        set_error("nep_nleigs_interpolation: degree %d needs cap >= %d", it.d, d1);
        return NEP_ERR_ARG;
    }
    for (int j = 0; j < d1; ++j) {
        if (sigma) { sigma[2 * j] = it.sigma[j].re; sigma[2 * j + 1] = it.sigma[j].im; }
        if (xi) { xi[2 * j] = it.xi[j].re; xi[2 * j + 1] = it.xi[j].im; }
        if (beta) beta[j] = it.beta[j];
        if (dd)
            for (int i = 0; i < nt; ++i) {
                dd[2 * (i + (size_t)nt * j)] = it.dd[i + (size_t)nt * j].re;
                dd[2 * (i + (size_t)nt * j) + 1] = it.dd[i + (size_t)nt * j].im;
            }
    }
    return NEP_OK;
}

extern "C" int nep_nleigs_solve(nep_split_t h, const nep_region* r, const nep_nleigs_opts* o, nep_result_t* out,
                                int32_t* degree, void* stream) {
    if (h && h->has_ext) {
        set_error("this entry point evaluates the functions on the device: not available with callback or table terms");
        return NEP_ERR_UNSUPPORTED;
    }
    if (!out) { set_error("out is NULL"); return NEP_ERR_ARG; }
    *out = nullptr;
    NleigsParams q;
    NEP_TRY(nleigs_params(h, r, o, &q));
    if (h->nterms > 8) { set_error("nleigs: at most 8 terms"); return NEP_ERR_UNSUPPORTED; }
    NleigsInterp it;
    NEP_TRY(nleigs_interpolation(h->nodes, h->coef, h->roots, mk(r->center_re, r->center_im), r->a, r->b, q.tol,
                                 q.dmax, q.nb, &it));
    if (degree) *degree = it.d;
    const size_t N = (size_t)it.d * h->n;
    const int kmax = (int)std::min<size_t>((size_t)q.kmax, N);
    std::vector<zd> start(N);
    draw_probe_block(q.seed, N, false, reinterpret_cast<double*>(start.data()));
    KsOpts ks;
    NEP_TRY(ks_params(q.max_restarts, q.keep, q.restart_tol, q.nev, kmax, q.exact, &ks));
    NleigsOut res;
    cudaStream_t st = (cudaStream_t)stream;
    NEP_TRY(nleigs_run(h->dev(), it, q.shift, kmax, reinterpret_cast<const double*>(start.data()),
                       mk(r->center_re, r->center_im), r->a, r->b, q.eig_tol, q.exact, &res, st, q.toar, ks));
    nep_result* rr = new nep_result();
    rr->n = h->n;
    rr->nconv = (int)res.lam.size();
    rr->m = 0;
    rr->flags = (it.converged ? 0 : NEP_WARN_INTERP) | (res.lu_info ? NEP_WARN_SINGULAR_NODE : 0);
    rr->info.n = h->n;
    rr->info.flags = rr->flags;
    rr->info.krylov_steps = res.steps;
    rr->info.restarts = res.restarts;
    for (size_t q2 = 0; q2 < res.lam.size(); ++q2) {
        rr->lam.push_back(res.lam[q2].re);
        rr->lam.push_back(res.lam[q2].im);
        rr->resid.push_back(res.eta[q2]);
    }
    for (const zd& v : res.X) {
        rr->X.push_back(v.re);
        rr->X.push_back(v.im);
    }
    *out = rr;
    return NEP_OK;
}

// ----------------------------------------------------------------- Interpol (Sec. 4.4)
// c[i + nt k] = 2/(d+1) sum_j f_i(lambda(nu_j)) cos(k omega_j), omega_j = (j + 1/2) pi / (d+1),
// nu_j = cos omega_j, lambda = a theta + center (Eqs. (interpolnu), (polinterpcoef))
static int interpol_coefs(const nep_split* h, const nep_region* r, int d, std::vector<zd>* c) {
    if (!r || !(r->a > 0) || !(r->b > 0)) { set_error("interpol: region semi-axes must be positive"); return NEP_ERR_ARG; }
    if (r->center_im != 0.0) { set_error("interpol: the interval is the real axis of a region with a real centre"); return NEP_ERR_ARG; }
    if (d < 2 || d > 63) { set_error("interpol: degree must be in 2 .. 63"); return NEP_ERR_ARG; }
    const int nt = h->nterms;
    std::vector<zd> lam(d + 1), F((size_t)nt * (d + 1));
    std::vector<double> om(d + 1);
    for (int j = 0; j <= d; ++j) {
        om[j] = (j + 0.5) * M_PI / (d + 1);
        lam[j] = mk(r->a * std::cos(om[j]) + r->center_re, 0.0);
    }
    NEP_TRY(host_terms(h, lam.data(), d + 1, F.data(), nullptr));
    c->assign((size_t)nt * (d + 1), mk(0.0, 0.0));
    for (int i = 0; i < nt; ++i)
        for (int k = 0; k <= d; ++k) {
            zd s = mk(0.0, 0.0);
            for (int j = 0; j <= d; ++j) s = s + std::cos(k * om[j]) * F[i + (size_t)nt * j];
            (*c)[i + (size_t)nt * k] = (2.0 / (d + 1)) * s;
        }
    return NEP_OK;
}

extern "C" int nep_interpol_coefficients(int32_t nterms, const nep_fn* f, const nep_region* r, int32_t degree,
                                         double* coef) {
    if (nterms < 1 || nterms > 32 || !f || !coef) { set_error("nep_interpol_coefficients: bad arguments"); return NEP_ERR_ARG; }
    nep_split h;  // the function trees only, on the host
    h.nterms = nterms;
    h.ext.resize(nterms);
    for (int i = 0; i < nterms; ++i) {
        if (f[i].kind == NEP_FN_CALLBACK || f[i].kind == NEP_FN_TABLE) {
            set_error("nep_interpol_coefficients: built-in function kinds only");
            return NEP_ERR_UNSUPPORTED;
        }
        const int root = flatten_fn(&h, &f[i], 0);
        if (root < 0) return NEP_ERR_ARG;
        h.roots.push_back(root);
    }
    std::vector<zd> c;
    NEP_TRY(interpol_coefs(&h, r, degree, &c));
    memcpy(coef, c.data(), sizeof(zd) * c.size());
    return NEP_OK;
}

extern "C" int nep_interpol_solve(nep_split_t h, const nep_region* r, const nep_interpol_opts* o, nep_result_t* out,
                                  void* stream) {
    if (!out) { set_error("out is NULL"); return NEP_ERR_ARG; }
    *out = nullptr;
    if (!h || !r) { set_error("null handle or region"); return NEP_ERR_ARG; }
    if (h->has_ext) {
        set_error("this entry point evaluates the functions on the device: not available with callback or table terms");
        return NEP_ERR_UNSUPPORTED;
    }
    if (h->nterms > 8) { set_error("interpol: at most 8 terms"); return NEP_ERR_UNSUPPORTED; }
    nep_interpol_opts z{};
    if (!o) o = &z;
    const int d = o->degree > 0 ? o->degree : 40;
    const int kry = o->krylov > 0 ? o->krylov : 60;
    const double eig_tol = o->eig_tol > 0 ? o->eig_tol : 1e-8;
    if (kry > 512) { set_error("interpol: krylov <= 512"); return NEP_ERR_ARG; }
    std::vector<zd> c;
    NEP_TRY(interpol_coefs(h, r, d, &c));
    for (int i = 0; i < h->nterms; ++i) {
        const int rc = check_region_node(h, h->roots[i], r, true);
        if (rc) return rc;
    }
    // the shift in theta: (lambda_shift - centre) / a
    const zd ls = o->has_shift ? mk(o->shift_re, o->shift_im) : mk(r->center_re, 0.0);
    const zd sigma = mk((ls.re - r->center_re) / r->a, ls.im / r->a);
    const size_t N = (size_t)d * h->n;
    const int kmax = (int)std::min<size_t>((size_t)kry, N);
    std::vector<zd> start(N);
    draw_probe_block(o->seed, N, false, reinterpret_cast<double*>(start.data()));
    KsOpts ks;
    NEP_TRY(ks_params(o->max_restarts, o->keep, o->restart_tol, o->nev, kmax, o->fast_solves == 0, &ks));
    NleigsOut res;
    cudaStream_t st = (cudaStream_t)stream;
    NEP_TRY(interpol_run(h->dev(), c, d, sigma, r->a, r->center_re, kmax, reinterpret_cast<const double*>(start.data()),
                         mk(r->center_re, r->center_im), r->a, r->b, eig_tol, o->fast_solves == 0, &res, st, ks));
    nep_result* rr = new nep_result();
    rr->n = h->n;
    rr->nconv = (int)res.lam.size();
    rr->m = 0;
    rr->flags = res.lu_info ? NEP_WARN_SINGULAR_NODE : 0;
    rr->info.n = h->n;
    rr->info.flags = rr->flags;
    rr->info.krylov_steps = res.steps;
    rr->info.restarts = res.restarts;
    for (size_t q2 = 0; q2 < res.lam.size(); ++q2) {
        rr->lam.push_back(res.lam[q2].re);
        rr->lam.push_back(res.lam[q2].im);
        rr->resid.push_back(res.eta[q2]);
    }
    for (const zd& v : res.X) {
        rr->X.push_back(v.re);
        rr->X.push_back(v.im);
    }
    *out = rr;
    return NEP_OK;
}

extern "C" int nep_plan_result(nep_plan_t p, nep_result_t* out) {
    if (!p || !out) { set_error("nep_plan_result: bad arguments"); return NEP_ERR_ARG; }
    const int n = p->h->n, N = p->Np, LM = p->LM;  // per-point arrays hold the solved points
    nep_result* r = new nep_result();
    r->n = n;
    r->m = p->m;
    std::vector<int> order(LM + 1, 0);
    NEP_CUDA(cudaMemcpy(order.data(), p->order, sizeof(int) * (p->m > 0 ? p->m + 1 : 1), cudaMemcpyDeviceToHost));
    const int nc = p->m > 0 && p->kb > 0 ? order[0] : 0;
    r->nconv = nc;
    std::vector<zd> lam(std::max(p->m, 1));
    std::vector<double> eta(std::max(p->m, 1));
    std::vector<int> ok(std::max(p->m, 1));
    if (p->m > 0 && p->kb > 0) {
        NEP_CUDA(cudaMemcpy(lam.data(), p->lamn, sizeof(zd) * p->m, cudaMemcpyDeviceToHost));
        NEP_CUDA(cudaMemcpy(eta.data(), p->eta, sizeof(double) * p->m, cudaMemcpyDeviceToHost));
        NEP_CUDA(cudaMemcpy(ok.data(), p->ok, sizeof(int) * p->m, cudaMemcpyDeviceToHost));
    }
    r->lam.resize(2 * (size_t)nc);
    r->resid.resize(nc);
    r->X.resize(2 * (size_t)n * nc);
    for (int q = 0; q < nc; ++q) {
        const int c = order[1 + q];
        r->lam[2 * q] = lam[c].re;
        r->lam[2 * q + 1] = lam[c].im;
        r->resid[q] = eta[c];
        NEP_CUDA(cudaMemcpy(r->X.data() + 2 * (size_t)n * q, p->Xc + (size_t)n * c, sizeof(zd) * n, cudaMemcpyDeviceToHost));
    }
    r->sigma.resize(LM);
    NEP_CUDA(cudaMemcpy(r->sigma.data(), p->sigma, sizeof(double) * LM, cudaMemcpyDeviceToHost));
    std::vector<double> beta(N);
    std::vector<int> sweeps(N), info(N);
    NEP_CUDA(cudaMemcpy(beta.data(), p->beta, sizeof(double) * N, cudaMemcpyDeviceToHost));
    NEP_CUDA(cudaMemcpy(sweeps.data(), p->sweeps, sizeof(int) * N, cudaMemcpyDeviceToHost));
    NEP_CUDA(cudaMemcpy(info.data(), p->info, sizeof(int) * N, cudaMemcpyDeviceToHost));
    int flags = 0, msw = 0;
    double mb = 0;
    for (int j = 0; j < N; ++j) {
        mb = std::max(mb, beta[j]);
        msw = std::max(msw, sweeps[j]);
        if (beta[j] > p->o.refine_tol) flags |= NEP_WARN_REFINE;
        if (info[j]) flags |= NEP_WARN_SINGULAR_NODE;
    }
    if (p->m == LM) flags |= NEP_WARN_SATURATED;
    r->pt_sweeps.assign(sweeps.begin(), sweeps.end());
    r->pt_info.assign(info.begin(), info.end());
    r->pt_beta = beta;
    int nfail = 0, nleft = 0;
    for (int c = 0; c < p->m && p->kb > 0; ++c) {
        nfail += ok[c] == 0;
        nleft += ok[c] == 2;
    }
    if (nfail) flags |= NEP_WARN_NEWTON;
    r->flags = flags;
    nep_result_info_t& in = r->info;
    in.n = n;
    in.N = p->N;
    in.L = p->L;
    in.M = p->M;
    in.precision = p->o.precision;
    in.hankel_rank = p->m;
    in.basis_rank = p->kb;
    in.ncandidates = p->m;
    in.max_sweeps = msw;
    in.svd_sweeps = p->svd_sweeps;
    in.flags = flags;
    in.max_backward = mb;
    in.newton_failed = nfail;
    in.newton_left = nleft;
    float t[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&t[i], p->ev[i], p->ev[i + 1]);
    in.ms_assemble = t[0];
    in.ms_factor = t[1];
    in.ms_solve = t[2];
    in.ms_moments = t[3];
    in.ms_extract = t[4];
    float tot = 0;
    cudaEventElapsedTime(&tot, p->ev[0], p->ev[5]);
    in.ms_total = tot;
    *out = r;
    return NEP_OK;
}

namespace nep {
void result_set_times(nep_result_t r, double queued_ms, double latency_ms) {
    if (!r) return;
    r->info.ms_queued = queued_ms;
    r->info.ms_latency = latency_ms;
}
}  // namespace nep

// Probe block drawn from a seed: a SplitMix64 stream and Box-Muller, Re and Im iid N(0,1)
// (Im = 0 when real_only, as conjugate-symmetric quadrature needs).
void nep::draw_probe_block(uint64_t seed, size_t count, bool real_only, double* out) {
    uint64_t state = seed;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto unif = [&]() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    for (size_t i = 0; i < count; ++i) {
        const double u1 = unif(), u2 = unif();
        const double rr = std::sqrt(-2.0 * std::log(u1));
        out[2 * i] = rr * std::cos(2 * M_PI * u2);
        out[2 * i + 1] = real_only ? 0.0 : rr * std::sin(2 * M_PI * u2);
    }
}

extern "C" int nep_ciss_solve(nep_split_t h, const nep_region* r, int32_t N, int32_t L, int32_t M, const nep_opts* o,
                              const double* V_host, nep_result_t* out) {
    if (!out) { set_error("out is NULL"); return NEP_ERR_ARG; }
    *out = nullptr;
    nep_plan_t p = nullptr;
    NEP_TRY(nep_plan_create(h, r, N, L, M, o, &p));
    const size_t nl = (size_t)h->n * L;
    std::vector<zd> V(nl);
    if (V_host) {
        memcpy(V.data(), V_host, sizeof(zd) * nl);
    } else {
        draw_probe_block(p->o.seed, nl, p->o.symmetric != 0, reinterpret_cast<double*>(V.data()));
    }
    int rc = NEP_OK;
    zd* dV = nullptr;
    if (cudaMalloc((void**)&dV, sizeof(zd) * nl) != cudaSuccess) rc = NEP_ERR_NOMEM;
    if (!rc && cudaMemcpy(dV, V.data(), sizeof(zd) * nl, cudaMemcpyHostToDevice) != cudaSuccess) rc = NEP_ERR_CUDA;
    if (!rc) rc = nep_plan_execute(p, dV, nullptr);
    if (!rc) rc = nep_plan_result(p, out);
    cudaFree(dV);
    nep_plan_destroy(p);
    return rc;
}

extern "C" int nep_result_get(nep_result_t r, int32_t* nconv, const double** lambda, const double** X,
                              const double** resid, int32_t* hankel_rank, int32_t* flags) {
    if (!r) { set_error("null result"); return NEP_ERR_ARG; }
    if (nconv) *nconv = r->nconv;
    if (lambda) *lambda = r->lam.data();
    if (X) *X = r->X.data();
    if (resid) *resid = r->resid.data();
    if (hankel_rank) *hankel_rank = r->m;
    if (flags) *flags = r->flags;
    return NEP_OK;
}

extern "C" int nep_result_points(nep_result_t r, int32_t* npts, const int32_t** sweeps, const int32_t** lu_info,
                                 const double** backward) {
    if (!r) { set_error("null result"); return NEP_ERR_ARG; }
    if (npts) *npts = (int32_t)r->pt_sweeps.size();
    if (sweeps) *sweeps = r->pt_sweeps.data();
    if (lu_info) *lu_info = r->pt_info.data();
    if (backward) *backward = r->pt_beta.data();
    return NEP_OK;
}

extern "C" int nep_result_info(nep_result_t r, nep_result_info_t* info) {
    if (!r || !info) { set_error("null result or info"); return NEP_ERR_ARG; }
    *info = r->info;
    return NEP_OK;
}

extern "C" int nep_result_hankel_sigma(nep_result_t r, const double** sigma, int32_t* count) {
    if (!r) { set_error("null result"); return NEP_ERR_ARG; }
    if (sigma) *sigma = r->sigma.data();
    if (count) *count = (int32_t)r->sigma.size();
    return NEP_OK;
}

extern "C" int nep_result_free(nep_result_t r) {
    delete r;
    return NEP_OK;
}

// ============================================================================ step entry points
extern "C" int nep_assemble_band(nep_split_t h, int32_t npts, const double* F_dev, int32_t precision, void* ab_dev,
                                 double* tnorm_dev, void* stream) {
    if (!h || !F_dev || !ab_dev || npts < 0) { set_error("nep_assemble_band: bad arguments"); return NEP_ERR_ARG; }
    const SplitDev s = h->dev();
    if (precision == NEP_PREC_MIXED)
        return launch_assemble<float>(s, npts, (const zd*)F_dev, (zf*)ab_dev, tnorm_dev, nullptr, (cudaStream_t)stream);
    if (precision == NEP_PREC_FP64)
        return launch_assemble<double>(s, npts, (const zd*)F_dev, (zd*)ab_dev, tnorm_dev, nullptr, (cudaStream_t)stream);
    set_error("bad precision");
    return NEP_ERR_ARG;
}

extern "C" int nep_band_factor(nep_split_t h, int32_t npts, int32_t precision, void* ab_dev, int32_t* ipiv_dev,
                               int32_t* info_dev, void* stream) {
    if (!h || !ab_dev || !ipiv_dev || !info_dev || npts < 0) { set_error("nep_band_factor: bad arguments"); return NEP_ERR_ARG; }
    const SplitDev s = h->dev();
    if (precision == NEP_PREC_MIXED) return launch_band_lu<float>(s, npts, (zf*)ab_dev, ipiv_dev, info_dev, nullptr, (cudaStream_t)stream);
    if (precision == NEP_PREC_FP64) return launch_band_lu<double>(s, npts, (zd*)ab_dev, ipiv_dev, info_dev, nullptr, (cudaStream_t)stream);
    set_error("bad precision");
    return NEP_ERR_ARG;
}

// The narrow-band sweeps read U by columns: the step entry point builds that copy in a
// stream-ordered temporary for the call.
template <typename T>
static int band_solve_step(const SplitDev& s, int npts, const cx<T>* ab, const int* ipiv, int L, cx<T>* B,
                           cudaStream_t st) {
    if (!band_sweeps_fit(s.kl, s.ku) || npts <= 0 || L <= 0)
        return launch_band_solve<T>(s, npts, ab, nullptr, ipiv, L, B, nullptr, st);
    cx<T>* ut = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&ut, sizeof(cx<T>) * (size_t)npts * s.n * (s.kl + s.ku + 1), st));
    int rc = band_transpose_u<T>(s, npts, ab, ut, st);
    if (!rc) rc = launch_band_solve<T>(s, npts, ab, ut, ipiv, L, B, nullptr, st);
    cudaFreeAsync(ut, st);
    return rc;
}

extern "C" int nep_band_solve(nep_split_t h, int32_t npts, int32_t precision, const void* ab_dev, const int32_t* ipiv_dev,
                              int32_t L, void* B_dev, void* stream) {
    if (!h || !ab_dev || !ipiv_dev || !B_dev || npts < 0 || L < 0) { set_error("nep_band_solve: bad arguments"); return NEP_ERR_ARG; }
    const SplitDev s = h->dev();
    if (precision != NEP_PREC_MIXED && precision != NEP_PREC_FP64) { set_error("bad precision"); return NEP_ERR_ARG; }
    return precision == NEP_PREC_MIXED
               ? band_solve_step<float>(s, npts, (const zf*)ab_dev, ipiv_dev, L, (zf*)B_dev, (cudaStream_t)stream)
               : band_solve_step<double>(s, npts, (const zd*)ab_dev, ipiv_dev, L, (zd*)B_dev, (cudaStream_t)stream);
}

extern "C" int nep_band_solve_adjoint(nep_split_t h, int32_t npts, int32_t precision, const void* ab_dev,
                                      const int32_t* ipiv_dev, int32_t L, void* B_dev, void* stream) {
    if (!h || !ab_dev || !ipiv_dev || !B_dev || npts < 0 || L < 0) {
        set_error("nep_band_solve_adjoint: bad arguments");
        return NEP_ERR_ARG;
    }
    const SplitDev s = h->dev();
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == NEP_PREC_MIXED)
        return launch_band_solve_adjoint<float>(s, npts, (const zf*)ab_dev, ipiv_dev, L, (zf*)B_dev, nullptr, st);
    if (precision == NEP_PREC_FP64)
        return launch_band_solve_adjoint<double>(s, npts, (const zd*)ab_dev, ipiv_dev, L, (zd*)B_dev, nullptr, st);
    set_error("bad precision");
    return NEP_ERR_ARG;
}

extern "C" int nep_band_transpose_u(nep_split_t h, int32_t npts, int32_t precision, const void* ab_dev, void* ut_dev,
                                    void* stream) {
    if (!h || !ab_dev || !ut_dev || npts < 0) { set_error("nep_band_transpose_u: bad arguments"); return NEP_ERR_ARG; }
    const SplitDev s = h->dev();
    if (precision == NEP_PREC_MIXED) return band_transpose_u<float>(s, npts, (const zf*)ab_dev, (zf*)ut_dev, (cudaStream_t)stream);
    if (precision == NEP_PREC_FP64) return band_transpose_u<double>(s, npts, (const zd*)ab_dev, (zd*)ut_dev, (cudaStream_t)stream);
    set_error("bad precision");
    return NEP_ERR_ARG;
}

extern "C" int nep_band_solve_cols(nep_split_t h, int32_t npts, int32_t precision, const void* ab_dev, const void* ut_dev,
                                   const int32_t* ipiv_dev, int32_t L, void* B_dev, void* stream) {
    if (!h || !ab_dev || !ipiv_dev || !B_dev || npts < 0 || L < 0) { set_error("nep_band_solve_cols: bad arguments"); return NEP_ERR_ARG; }
    const SplitDev s = h->dev();
    if (band_sweeps_fit(s.kl, s.ku) && !ut_dev) {
        set_error("nep_band_solve_cols: this band needs the column copy of U (nep_band_transpose_u)");
        return NEP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == NEP_PREC_MIXED)
        return launch_band_solve<float>(s, npts, (const zf*)ab_dev, (const zf*)ut_dev, ipiv_dev, L, (zf*)B_dev, nullptr, st);
    if (precision == NEP_PREC_FP64)
        return launch_band_solve<double>(s, npts, (const zd*)ab_dev, (const zd*)ut_dev, ipiv_dev, L, (zd*)B_dev, nullptr, st);
    set_error("bad precision");
    return NEP_ERR_ARG;
}

extern "C" int nep_split_residual(nep_split_t h, int32_t npts, const double* F_dev, int32_t L, const double* V_dev,
                                  const double* Y_dev, double* R_dev, void* stream) {
    if (!h || !F_dev || !V_dev || !Y_dev || !R_dev || npts < 0 || L < 1) { set_error("nep_split_residual: bad arguments"); return NEP_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const SplitDev s = h->dev();
    zd* tval = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&tval, sizeof(zd) * (size_t)std::max(npts, 1) * std::max<int64_t>(h->nnz, 1), st));
    int rc = launch_assemble<double>(s, npts, (const zd*)F_dev, nullptr, nullptr, tval, st);
    if (!rc) rc = launch_split_residual(s, npts, tval, L, (const zd*)V_dev, (const zd*)Y_dev, (zd*)R_dev, nullptr, nullptr, st);
    cudaFreeAsync(tval, st);
    return rc;
}

extern "C" int nep_moments(int32_t n, int32_t L, int32_t N, int32_t K, const double* coef_dev, const double* Y_dev,
                           double* S_dev, void* stream) {
    if (n < 1 || L < 1 || N < 1 || K < 1 || !coef_dev || !Y_dev || !S_dev) { set_error("nep_moments: bad arguments"); return NEP_ERR_ARG; }
    return launch_moments(n, L, N, K, (const zd*)coef_dev, (const zd*)Y_dev, (zd*)S_dev, (cudaStream_t)stream);
}

extern "C" int nep_jacobi_svd(int32_t rows, int32_t cols, double* A_dev, double* W_dev, double* sigma_dev, void* stream) {
    if (rows < cols || cols < 1 || !A_dev || !W_dev || !sigma_dev) { set_error("nep_jacobi_svd: need rows >= cols >= 1"); return NEP_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    JacobiWork w{};
    zd* U = nullptr;
    NEP_CUDA(cudaMallocAsync((void**)&w.Vm, sizeof(zd) * (size_t)cols * cols, st));
    NEP_CUDA(cudaMallocAsync((void**)&w.flags, 2 * sizeof(int), st));
    NEP_CUDA(cudaMallocAsync((void**)&w.sweeps, sizeof(int), st));
    NEP_CUDA(cudaMallocAsync((void**)&w.bar, 2 * sizeof(unsigned), st));
    NEP_CUDA(cudaMallocAsync((void**)&w.err, sizeof(int), st));
    NEP_CUDA(cudaMallocAsync((void**)&U, sizeof(zd) * (size_t)rows * cols, st));
    NEP_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    int rc = jacobi_svd(rows, cols, (zd*)A_dev, U, (zd*)W_dev, sigma_dev, w, st);
    int err = 0;
    if (!rc) {
        if (cudaMemcpyAsync(A_dev, U, sizeof(zd) * (size_t)rows * cols, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = NEP_ERR_CUDA;
    }
    cudaFreeAsync(w.Vm, st);
    cudaFreeAsync(w.flags, st);
    cudaFreeAsync(w.sweeps, st);
    cudaFreeAsync(w.bar, st);
    cudaFreeAsync(w.err, st);
    cudaFreeAsync(U, st);
    if (!rc && err) { set_error("grid barrier timed out"); rc = NEP_ERR_INTERNAL; }
    return rc;
}

extern "C" int nep_small_eig(int32_t m, const double* A_dev, double* eval_dev, double* evec_dev, void* stream) {
    if (m < 1 || !A_dev || !eval_dev) { set_error("nep_small_eig: bad arguments"); return NEP_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    void* g = nullptr;
    NEP_CUDA(cudaMallocAsync(&g, sizeof(zd) * ((size_t)2 * m * (m + 1) + m) + 256, st));
    int rc = small_eig<double>(m, (const zd*)A_dev, (zd*)eval_dev, (zd*)evec_dev, nullptr, g, st);
    cudaFreeAsync(g, st);
    return rc;
}
