// phc_api.cpp -- host side of the C ABI declared in include/phc.h:
// argument checks, compilation of coefficient/exponent lists into the
// device term tables, the embedding of Section 2.1, and the launch sequence
// (track -> classify [-> drop z_k]) of each entry point.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "phc_internal.h"

using phc::DevTables;
using phc::TermRec;

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) return fail(PHC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
    } while (0)

extern "C" const char *phc_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ options

extern "C" int phc_default_opts(phc_opts *o)
{
    if (!o) return fail(PHC_EINVAL, "opts is NULL");
    std::memset(o, 0, sizeof *o);
    o->h_init = 0.01;
    o->h_max = 0.1;
    o->h_min = 1e-14;
    o->expand_after = 3;
    o->expand = 2.0;
    o->shrink = 0.5;
    o->max_corr_iters = 3;
    o->corr_tol = 1e-9;
    o->corr_contract = 0.5;
    o->max_steps = 20000;
    o->max_steps_decade = 300;
    o->diverge_norm = 1e6;
    o->endpoint_inf_norm = 1e4;
    o->end_zone = 0.9;
    o->growth_inf = 1.1220184543019633;  // 10^0.05
    o->end_iters = 8;
    o->end_tol = 1e-13;
    o->cond_regular = 1e6;
    o->res_regular = 1e-12;
    o->slack_tol = 1e-8;
    o->precision = PHC_PREC_FP64;
    o->fp32_t_max = 0.9;
    o->fp32_pivot_ratio = 1e4;
    o->block_threads = 0;
    o->max_blocks = 0;
    o->tail_drain = 0.8;
    o->tail_threads = 0;
    o->compact = 1;
    o->group_paths = 0;
    return PHC_OK;
}

static int check_opts(const phc_opts &o)
{
    if (!(o.h_init > 0 && o.h_max > 0 && o.h_min > 0 && o.h_min <= o.h_max))
        return fail(PHC_EINVAL, "step sizes must satisfy 0 < h_min <= h_max and h_init > 0");
    if (o.expand_after < 1 || !(o.expand >= 1.0) || !(o.shrink > 0.0 && o.shrink < 1.0))
        return fail(PHC_EINVAL, "invalid step control (expand_after >= 1, expand >= 1, 0 < shrink < 1)");
    if (o.max_corr_iters < 1 || o.max_corr_iters > 64 || o.end_iters < 0 || o.end_iters > 64)
        return fail(PHC_EINVAL, "iteration counts out of range");
    if (o.max_steps < 1 || o.max_steps_decade < 1) return fail(PHC_EINVAL, "step budgets must be positive");
    if (!(o.growth_inf >= 1.0)) return fail(PHC_EINVAL, "growth_inf must be >= 1");
    if (o.precision != PHC_PREC_FP64 && o.precision != PHC_PREC_FP32_INTERIOR)
        return fail(PHC_EINVAL, "unknown precision %d", o.precision);
    if (!(o.fp32_pivot_ratio >= 1.0)) return fail(PHC_EINVAL, "fp32_pivot_ratio must be >= 1");
    if (o.block_threads < 0 || o.block_threads % 32) return fail(PHC_EINVAL, "block_threads must be a multiple of 32");
    if (!(o.tail_drain >= 0.0 && o.tail_drain <= 1.0)) return fail(PHC_EINVAL, "tail_drain must be in [0, 1]");
    if (o.tail_threads != 0 && o.tail_threads != 8 && o.tail_threads != 16 && o.tail_threads != 32)
        return fail(PHC_EINVAL, "tail_threads must be 0, 8, 16 or 32");
    if (o.compact != 0 && o.compact != 1) return fail(PHC_EINVAL, "compact must be 0 or 1");
    if (o.group_paths < -1 || o.group_paths > 1) return fail(PHC_EINVAL, "group_paths must be -1, 0 or 1");
    return PHC_OK;
}

// ------------------------------------------------------------------ handles

struct DeviceTable {
    DevTables view{};
    void *blob = nullptr;
};

struct phc_homotopy {
    int n = 0;
    int n_sys = 1;              // systems sharing the supports (batch handle)
    // host copy of the system lists (coefficients of system 0 for a batch)
    std::vector<int32_t> tpe;
    std::vector<uint8_t> exps;
    std::vector<phc_cd> coefs;
    phc_cd gamma{1.0, 0.0};
    std::vector<int32_t> deg;
    int64_t paths_per_system = 0;
    int64_t num_paths = 0;
    // device
    int device = 0;
    DeviceTable total;    // total-degree homotopy
    DeviceTable cascade;  // cascade stage (last slack), built on first use
    // coefficient-parameter homotopy (phc_make_parameter_homotopy): no
    // total-degree start system; `total` holds (gamma c_start, c_target -
    // gamma c_start) per term and `target` (c_target, 0), the exact target
    // for the classification and refinement at t = 1
    int parameter = 0;
    DeviceTable target;
    // polyhedral homotopies (phc_make_polyhedral_homotopy): `total` holds
    // (0, c) per term of g (so t = 1 gives g for classification and
    // refinement); the cells' data live in one device block
    int polyhedral = 0;
    int n_cells = 0;
    void *d_poly = nullptr;
    const int64_t *d_path_off = nullptr;
    const double *d_powers = nullptr;
    const int64_t *d_H = nullptr, *d_U = nullptr;
    const int32_t *d_pairs = nullptr;
    int32_t *d_deg = nullptr, *d_root_off = nullptr;
    double2 *d_roots = nullptr;
    // scratch
    unsigned long long *d_qhead = nullptr;
    phc_path_stats *d_stats = nullptr;
    int64_t stats_cap = 0;
    phc_path_stats *d_stats2 = nullptr;
    int64_t stats2_cap = 0;
    double2 *d_xfull = nullptr;
    int64_t xfull_cap = 0;
    phc::Handoff *d_handoff = nullptr;  // paths moved to the tail kernel
    int64_t handoff_cap = 0;
    unsigned long long *d_tailc = nullptr;  // hand-off, idle and tail queue counters
};

static void free_table(DeviceTable &t)
{
    if (t.blob) cudaFree(t.blob);
    t.blob = nullptr;
}

// Terms of a homotopy with coefficients linear in t, as host vectors.
struct HostTerms {
    std::vector<TermRec> recs;
    std::vector<uint8_t> vars, exps;
    std::vector<double2> c0, c1;

    void add(int eq, const uint8_t *a, int n, double2 c0v, double2 c1v)
    {
        TermRec r{};
        r.eq = (uint8_t)eq;
        r.off = (uint16_t)vars.size();
        int k = 0;
        for (int j = 0; j < n; j++) {
            if (a[j] == 0) continue;
            vars.push_back((uint8_t)j);
            exps.push_back(a[j]);
            if (a[j] > 1) r.flags |= phc::TERM_POWERS;
            k++;
        }
        r.k = (uint8_t)k;
        recs.push_back(r);
        c0.push_back(c0v);
        c1.push_back(c1v);
    }
    // coefficients of one more system of a batch (same structure)
    void add_coef(double2 c0v, double2 c1v)
    {
        c0.push_back(c0v);
        c1.push_back(c1v);
    }
};

// Uploads go through a private non-blocking stream so that building a
// homotopy never waits for (or blocks) work the caller runs on its streams.
static int upload_table(const HostTerms &ht, int n, DeviceTable &out, cudaStream_t ps)
{
    const size_t T = ht.recs.size(), V = ht.vars.size();
    const size_t C = ht.c0.size();  // T per system
    const int n_sys = (int)(C / T);
    if (V > 65535) return fail(PHC_EUNSUPPORTED, "system too large (%zu exponent entries)", V);
    for (size_t q = 1; q < T; q++)
        if (ht.recs[q].eq < ht.recs[q - 1].eq) return fail(PHC_EINVAL, "internal: terms not grouped by equation");
    const size_t o_terms = 0;
    const size_t o_vars = o_terms + T * sizeof(TermRec);
    const size_t o_exps = o_vars + V;
    size_t o_c0 = o_exps + V;
    o_c0 = (o_c0 + 15) & ~(size_t)15;
    const size_t o_c1 = o_c0 + C * sizeof(double2);
    const size_t o_c0f = o_c1 + C * sizeof(double2);
    const size_t o_c1f = o_c0f + C * sizeof(float2);
    const size_t bytes = o_c1f + C * sizeof(float2);
    std::vector<char> host(bytes, 0);
    std::memcpy(host.data() + o_terms, ht.recs.data(), T * sizeof(TermRec));
    if (V) {
        std::memcpy(host.data() + o_vars, ht.vars.data(), V);
        std::memcpy(host.data() + o_exps, ht.exps.data(), V);
    }
    std::memcpy(host.data() + o_c0, ht.c0.data(), C * sizeof(double2));
    std::memcpy(host.data() + o_c1, ht.c1.data(), C * sizeof(double2));
    {
        float2 *f0 = reinterpret_cast<float2 *>(host.data() + o_c0f);
        float2 *f1 = reinterpret_cast<float2 *>(host.data() + o_c1f);
        for (size_t i = 0; i < C; i++) {
            f0[i] = make_float2((float)ht.c0[i].x, (float)ht.c0[i].y);
            f1[i] = make_float2((float)ht.c1[i].x, (float)ht.c1[i].y);
        }
    }
    void *blob = nullptr;
    if (cudaMalloc(&blob, bytes) != cudaSuccess) return fail(PHC_ENOMEM, "cudaMalloc of %zu table bytes", bytes);
    if (cudaMemcpyAsync(blob, host.data(), bytes, cudaMemcpyHostToDevice, ps) != cudaSuccess ||
        cudaStreamSynchronize(ps) != cudaSuccess) {
        cudaFree(blob);
        return fail(PHC_ECUDA, "upload of the term table");
    }
    char *b = static_cast<char *>(blob);
    out.blob = blob;
    out.view.n = n;
    out.view.n_terms = (int)T;
    out.view.n_ve = (int)V;
    out.view.n_sys = n_sys;
    out.view.f32 = 1;  // launchers of double precision work clear it
    out.view.coef_smem = 1;
    out.view.terms = reinterpret_cast<const TermRec *>(b + o_terms);
    out.view.vars = reinterpret_cast<const uint8_t *>(b + o_vars);
    out.view.exps = reinterpret_cast<const uint8_t *>(b + o_exps);
    out.view.c0 = reinterpret_cast<const double2 *>(b + o_c0);
    out.view.c1 = reinterpret_cast<const double2 *>(b + o_c1);
    out.view.c0f = reinterpret_cast<const float2 *>(b + o_c0f);
    out.view.c1f = reinterpret_cast<const float2 *>(b + o_c1f);
    return PHC_OK;
}

static int validate_lists(int n_eq, int n_var, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs,
                          bool square, std::vector<int32_t> *deg_out)
{
    if (n_var < 1 || n_var > PHC_MAX_VARS) return fail(PHC_EINVAL, "n_var = %d outside 1..%d", n_var, PHC_MAX_VARS);
    if (square && n_eq != n_var) return fail(PHC_EINVAL, "system is not square (%d equations, %d unknowns)", n_eq, n_var);
    if (n_eq < 1 || n_eq > 255) return fail(PHC_EINVAL, "n_eq = %d out of range", n_eq);
    if (!tpe || !exps || !coefs) return fail(PHC_EINVAL, "NULL list");
    std::vector<int32_t> deg(n_eq, 0);
    int64_t off = 0;
    for (int i = 0; i < n_eq; i++) {
        if (tpe[i] < 1) return fail(PHC_EINVAL, "equation %d has no terms", i);
        if (tpe[i] > 4096) return fail(PHC_EUNSUPPORTED, "equation %d has %d terms", i, tpe[i]);
        for (int k = 0; k < tpe[i]; k++, off++) {
            const phc_cd c = coefs[off];
            if (!std::isfinite(c.re) || !std::isfinite(c.im))
                return fail(PHC_EINVAL, "coefficient %lld of equation %d is not finite", (long long)off, i);
            int d = 0;
            for (int j = 0; j < n_var; j++) d += exps[off * n_var + j];
            if (d > deg[i]) deg[i] = d;
        }
        if (deg[i] < 1) return fail(PHC_EINVAL, "equation %d has degree 0", i);
    }
    if (deg_out) *deg_out = deg;
    return PHC_OK;
}

extern "C" int phc_make_homotopy_batch(int n_eq, int n_var, const int32_t *tpe, const uint8_t *exps, int n_sys,
                                       const phc_cd *coefs, const phc_cd *gammas, phc_homotopy **out)
try {
    if (!out) return fail(PHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_sys < 1) return fail(PHC_EINVAL, "n_systems = %d < 1", n_sys);
    if (!gammas) return fail(PHC_EINVAL, "gammas is NULL");
    std::vector<int32_t> deg;
    int rc = validate_lists(n_eq, n_var, tpe, exps, coefs, true, &deg);
    if (rc) return rc;
    const int n = n_var;
    int64_t T = 0;
    for (int i = 0; i < n_eq; i++) T += tpe[i];
    for (int s = 0; s < n_sys; s++) {
        const phc_cd g = gammas[s];
        if (!std::isfinite(g.re) || !std::isfinite(g.im) || (g.re == 0.0 && g.im == 0.0))
            return fail(PHC_EINVAL, "gamma of system %d must be finite and nonzero", s);
        for (int64_t k = 0; k < T; k++) {
            const phc_cd c = coefs[s * T + k];
            if (!std::isfinite(c.re) || !std::isfinite(c.im))
                return fail(PHC_EINVAL, "coefficient %lld of system %d is not finite", (long long)k, s);
        }
    }

    phc_homotopy *h = new (std::nothrow) phc_homotopy();
    if (!h) return fail(PHC_ENOMEM, "host allocation");
    h->n = n;
    h->n_sys = n_sys;
    h->tpe.assign(tpe, tpe + n_eq);
    h->exps.assign(exps, exps + T * n);
    h->coefs.assign(coefs, coefs + T);
    h->gamma = gammas[0];
    h->deg = deg;
    h->paths_per_system = 1;
    for (int i = 0; i < n; i++) {
        if (h->paths_per_system > (int64_t)1 << 40) {
            delete h;
            return fail(PHC_EUNSUPPORTED, "Bezout number too large");
        }
        h->paths_per_system *= deg[i];
    }
    h->num_paths = h->paths_per_system * n_sys;
    cudaGetDevice(&h->device);

    // total-degree homotopy: f terms (0, c); x_i^{d_i}: (gamma, -gamma); -1: (-gamma, gamma)
    HostTerms ht;
    for (int s = 0; s < n_sys; s++) {
        const phc_cd gamma = gammas[s];
        const phc_cd *cs = coefs + s * T;
        int64_t off = 0;
        for (int i = 0; i < n; i++) {
            for (int k = 0; k < tpe[i]; k++, off++) {
                const double2 c0 = make_double2(0.0, 0.0), c1 = make_double2(cs[off].re, cs[off].im);
                if (s == 0) ht.add(i, exps + off * n, n, c0, c1);
                else ht.add_coef(c0, c1);
            }
            const double2 g0 = make_double2(gamma.re, gamma.im), g1 = make_double2(-gamma.re, -gamma.im);
            if (s == 0) {
                std::vector<uint8_t> a(n, 0);
                a[i] = (uint8_t)deg[i];
                ht.add(i, a.data(), n, g0, g1);
                std::vector<uint8_t> z(n, 0);
                ht.add(i, z.data(), n, g1, g0);
            } else {
                ht.add_coef(g0, g1);
                ht.add_coef(g1, g0);
            }
        }
    }
    cudaStream_t ps = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return fail(PHC_ECUDA, "cudaStreamCreateWithFlags");
    }
    rc = upload_table(ht, n, h->total, ps);
    if (rc) {
        cudaStreamDestroy(ps);
        delete h;
        return rc;
    }
    // start system: degrees and the table of roots of unity
    std::vector<int32_t> roff(n);
    int total = 0;
    for (int i = 0; i < n; i++) {
        roff[i] = total;
        total += deg[i];
    }
    if (cudaMalloc(&h->d_deg, n * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&h->d_root_off, n * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&h->d_roots, total * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&h->d_qhead, sizeof(unsigned long long)) != cudaSuccess) {
        cudaStreamDestroy(ps);
        phc_destroy_homotopy(h);
        return fail(PHC_ENOMEM, "cudaMalloc of the start tables");
    }
    cudaError_t e = cudaMemcpyAsync(h->d_deg, deg.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_root_off, roff.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess) e = phc::launch_roots(h->d_deg, h->d_root_off, h->d_roots, n, total, ps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    cudaStreamDestroy(ps);
    if (e != cudaSuccess) {
        phc_destroy_homotopy(h);
        return fail(PHC_ECUDA, "start tables: %s", cudaGetErrorString(e));
    }
    *out = h;
    return PHC_OK;
} catch (...) {
    return fail(PHC_ENOMEM, "phc_make_homotopy_batch: host allocation failed");
}

extern "C" int phc_make_homotopy(int n_eq, int n_var, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs,
                                 phc_cd gamma, phc_homotopy **out)
{
    return phc_make_homotopy_batch(n_eq, n_var, tpe, exps, 1, coefs, &gamma, out);
}

extern "C" int phc_make_parameter_homotopy(int n_eq, int n_var, const int32_t *tpe, const uint8_t *exps,
                                           int n_sys, const phc_cd *coefs_start, const phc_cd *coefs_target,
                                           phc_cd gamma, phc_homotopy **out)
try {
    if (!out) return fail(PHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_sys < 1) return fail(PHC_EINVAL, "n_systems = %d < 1", n_sys);
    if (!coefs_start || !coefs_target) return fail(PHC_EINVAL, "NULL coefficients");
    std::vector<int32_t> deg;
    int rc = validate_lists(n_eq, n_var, tpe, exps, coefs_target, true, &deg);
    if (rc) return rc;
    if (!std::isfinite(gamma.re) || !std::isfinite(gamma.im) || (gamma.re == 0.0 && gamma.im == 0.0))
        return fail(PHC_EINVAL, "gamma must be finite and nonzero");
    const int n = n_var;
    int64_t T = 0;
    for (int i = 0; i < n_eq; i++) T += tpe[i];
    for (int64_t k = 0; k < T; k++)
        if (!std::isfinite(coefs_start[k].re) || !std::isfinite(coefs_start[k].im))
            return fail(PHC_EINVAL, "start coefficient %lld is not finite", (long long)k);
    for (int64_t k = 0; k < (int64_t)n_sys * T; k++)
        if (!std::isfinite(coefs_target[k].re) || !std::isfinite(coefs_target[k].im))
            return fail(PHC_EINVAL, "target coefficient %lld is not finite", (long long)k);

    phc_homotopy *h = new (std::nothrow) phc_homotopy();
    if (!h) return fail(PHC_ENOMEM, "host allocation");
    h->n = n;
    h->n_sys = n_sys;
    h->parameter = 1;
    h->tpe.assign(tpe, tpe + n_eq);
    h->exps.assign(exps, exps + T * n);
    h->coefs.assign(coefs_target, coefs_target + T);
    h->gamma = gamma;
    h->deg = deg;
    h->paths_per_system = 0;
    h->num_paths = 0;
    cudaGetDevice(&h->device);
    // (1-t) gamma g + t f: per term (gamma c_start, c_target - gamma c_start)
    HostTerms ht, hf;
    const double2 g = make_double2(gamma.re, gamma.im);
    for (int s = 0; s < n_sys; s++) {
        int64_t off = 0;
        for (int i = 0; i < n; i++) {
            for (int k = 0; k < tpe[i]; k++, off++) {
                const phc_cd cs = coefs_start[off], ct = coefs_target[(int64_t)s * T + off];
                const double2 c0 = make_double2(g.x * cs.re - g.y * cs.im, g.x * cs.im + g.y * cs.re);
                const double2 c1 = make_double2(ct.re - c0.x, ct.im - c0.y);
                const double2 f0 = make_double2(ct.re, ct.im), zero = make_double2(0.0, 0.0);
                if (s == 0) {
                    ht.add(i, exps + off * n, n, c0, c1);
                    hf.add(i, exps + off * n, n, f0, zero);
                } else {
                    ht.add_coef(c0, c1);
                    hf.add_coef(f0, zero);
                }
            }
        }
    }
    cudaStream_t ps = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return fail(PHC_ECUDA, "cudaStreamCreateWithFlags");
    }
    rc = upload_table(ht, n, h->total, ps);
    if (!rc) rc = upload_table(hf, n, h->target, ps);
    cudaStreamDestroy(ps);
    if (!rc && cudaMalloc(&h->d_qhead, sizeof(unsigned long long)) != cudaSuccess)
        rc = fail(PHC_ENOMEM, "cudaMalloc of the path counter");
    if (rc) {
        phc_destroy_homotopy(h);
        return rc;
    }
    *out = h;
    return PHC_OK;
} catch (...) {
    return fail(PHC_ENOMEM, "phc_make_parameter_homotopy: host allocation failed");
}

extern "C" void phc_destroy_homotopy(phc_homotopy *h)
{
    if (!h) return;
    free_table(h->total);
    free_table(h->cascade);
    free_table(h->target);
    if (h->d_deg) cudaFree(h->d_deg);
    if (h->d_root_off) cudaFree(h->d_root_off);
    if (h->d_roots) cudaFree(h->d_roots);
    if (h->d_qhead) cudaFree(h->d_qhead);
    if (h->d_stats) cudaFree(h->d_stats);
    if (h->d_stats2) cudaFree(h->d_stats2);
    if (h->d_xfull) cudaFree(h->d_xfull);
    if (h->d_handoff) cudaFree(h->d_handoff);
    if (h->d_tailc) cudaFree(h->d_tailc);
    if (h->d_poly) cudaFree(h->d_poly);
    delete h;
}

extern "C" int phc_tail_paths(const phc_homotopy *h, void *stream, int64_t *out, int64_t *units_out)
{
    if (!h || !out) return fail(PHC_EINVAL, "NULL argument");
    *out = 0;
    if (units_out) *units_out = 0;
    if (!h->d_tailc) return PHC_OK;
    unsigned long long v[4] = {0, 0, 0, 0};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CU(cudaMemcpyAsync(v, h->d_tailc, sizeof v, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *out = (int64_t)v[0];
    if (units_out) *units_out = (int64_t)v[3];
    return PHC_OK;
}

extern "C" int phc_num_paths(const phc_homotopy *h, int64_t *out)
{
    if (!h || !out) return fail(PHC_EINVAL, "NULL argument");
    *out = h->num_paths;
    return PHC_OK;
}

extern "C" int phc_sizeof_opts(void) { return (int)sizeof(phc_opts); }
extern "C" int phc_sizeof_stats(void) { return (int)sizeof(phc_path_stats); }

// ------------------------------------------------------------------ scratch

// The handle's scratch grows on the stream of the call that needs it
// (stream-ordered free and allocation: no device-wide synchronisation, so a
// call that grows it does not wait for work on other streams).
static int grow(void **ptr, int64_t *cap, int64_t want, size_t elem, cudaStream_t s, const char *what)
{
    if (*cap >= want) return PHC_OK;
    if (*ptr) cudaFreeAsync(*ptr, s);
    *ptr = nullptr;
    *cap = 0;
    if (cudaMallocAsync(ptr, (size_t)want * elem, s) != cudaSuccess)
        return fail(PHC_ENOMEM, "cudaMallocAsync of %lld %s", (long long)want, what);
    *cap = want;
    return PHC_OK;
}

static int ensure_stats(phc_homotopy *h, int64_t n, cudaStream_t s)
{
    return grow(reinterpret_cast<void **>(&h->d_stats), &h->stats_cap, n, sizeof(phc_path_stats), s, "path records");
}

static int ensure_handoff(phc_homotopy *h, int64_t lanes, cudaStream_t s)
{
    if (!h->d_tailc && cudaMallocAsync(reinterpret_cast<void **>(&h->d_tailc), 4 * sizeof(unsigned long long), s) !=
                           cudaSuccess)
        return fail(PHC_ENOMEM, "cudaMallocAsync of the tail counters");
    return grow(reinterpret_cast<void **>(&h->d_handoff), &h->handoff_cap, lanes, sizeof(phc::Handoff), s,
                "hand-off records");
}

static int ensure_xfull(phc_homotopy *h, int64_t elems, cudaStream_t s)
{
    return grow(reinterpret_cast<void **>(&h->d_xfull), &h->xfull_cap, elems, sizeof(double2), s, "endpoint values");
}

// ------------------------------------------------------------------ tracking

// The table the endpoints are classified and refined with: the homotopy at
// t = 1 (for a parameter homotopy its exact target).
static const DevTables &end_table(const phc_homotopy *h)
{
    return h->parameter ? h->target.view : h->total.view;
}

static int run_track(phc_homotopy *h, const DevTables &tab, int start_mode, const double2 *starts, int64_t first,
                     int64_t n, const phc_opts &o, double2 *x_out, int8_t *cls_out, phc_path_stats *stats,
                     cudaStream_t s, const int8_t *sel_cls = nullptr, const uint8_t *sel_sz = nullptr,
                     int64_t starts_per_system = 0, const DevTables *cls_tab = nullptr)
{
    CU(cudaMemsetAsync(h->d_qhead, 0, sizeof(unsigned long long), s));
    phc::TrackLaunch L{};
    L.tab = tab;
    L.tab.f32 = o.precision == PHC_PREC_FP32_INTERIOR;
    L.start_mode = start_mode;
    L.deg = h->d_deg;
    L.root_off = h->d_root_off;
    L.roots = h->d_roots;
    L.starts = starts;
    L.sel_cls = sel_cls;
    L.sel_sz = sel_sz;
    L.first = first;
    L.n_paths = n;
    L.paths_per_system = h->paths_per_system > 0 ? h->paths_per_system : 1;
    L.starts_per_system = starts_per_system;
    L.compact = o.compact;
    L.x_out = x_out;
    L.stats = stats;
    L.qhead = h->d_qhead;
    L.o = o;
    const bool tail = o.tail_drain > 0.0 && phc::tail_supported(L.tab);
    if (tail) {
        const int64_t lanes = phc::track_lanes(L, o.block_threads, o.max_blocks);
        if (lanes < 1) return fail(PHC_EUNSUPPORTED, "no launch configuration for %d unknowns", tab.n);
        int rc = ensure_handoff(h, lanes, s);
        if (rc) return rc;
        CU(cudaMemsetAsync(h->d_tailc, 0, 4 * sizeof(unsigned long long), s));
        L.handoff = h->d_handoff;
        L.handoff_n = h->d_tailc;
        L.idle_n = h->d_tailc + 1;
        L.tail_q = h->d_tailc + 2;
        L.tail_units = h->d_tailc + 3;
        L.drain_frac = o.tail_drain;
    } else if (h->d_tailc) {
        CU(cudaMemsetAsync(h->d_tailc, 0, 4 * sizeof(unsigned long long), s));  // phc_tail_paths reports 0
    }
    cudaError_t e = phc::launch_track(L, o.block_threads, o.max_blocks, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "track kernel launch: %s", cudaGetErrorString(e));
    if (tail) {
        e = phc::launch_tail(L, o.max_blocks, s);
        if (e != cudaSuccess) return fail(PHC_ECUDA, "tail kernel launch: %s", cudaGetErrorString(e));
    }
    phc::ClassifyLaunch C{};
    C.tab = cls_tab ? *cls_tab : tab;
    C.tab.f32 = 0;
    C.n_paths = n;
    C.x = x_out;
    C.stats = stats;
    C.cls = cls_out;
    C.o = o;
    e = phc::launch_classify(C, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "classify kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

extern "C" int phc_track_paths(phc_homotopy *h, int64_t first, int64_t n, const phc_opts *opts, phc_cd *x_out,
                               int8_t *cls_out, phc_path_stats *stats_out, void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (h->parameter && n > 0)
        return fail(PHC_EINVAL, "a parameter homotopy has no total-degree start system (use phc_track_from)");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle is tracked by phc_track_polyhedral");
    if (n < 0 || first < 0 || first + n > h->num_paths)
        return fail(PHC_EINVAL, "path range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)h->num_paths);
    if (n == 0) return PHC_OK;
    if (!x_out || !cls_out) return fail(PHC_EINVAL, "NULL output array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
        st = h->d_stats;
    }
    return run_track(h, h->total.view, 0, nullptr, first, n, o, reinterpret_cast<double2 *>(x_out), cls_out, st,
                     static_cast<cudaStream_t>(stream));
}

extern "C" int phc_track_from(phc_homotopy *h, const phc_cd *starts, int64_t n, int64_t starts_per_system,
                              const phc_opts *opts, phc_cd *x_out, int8_t *cls_out, phc_path_stats *stats_out,
                              void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle is tracked by phc_track_polyhedral");
    if (n < 0 || starts_per_system < 0) return fail(PHC_EINVAL, "n_starts or starts_per_system < 0");
    if (n == 0) return PHC_OK;
    if (!starts || !x_out || !cls_out) return fail(PHC_EINVAL, "NULL array");
    const int64_t systems = starts_per_system > 0 ? (n + starts_per_system - 1) / starts_per_system : 1;
    if (systems > h->n_sys)
        return fail(PHC_EINVAL, "%lld starts at %lld per system need %lld systems, the handle has %d", (long long)n,
                    (long long)starts_per_system, (long long)systems, h->n_sys);
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
        st = h->d_stats;
    }
    return run_track(h, h->total.view, 1, reinterpret_cast<const double2 *>(starts), 0, n, o,
                     reinterpret_cast<double2 *>(x_out), cls_out, st, static_cast<cudaStream_t>(stream), nullptr,
                     nullptr, starts_per_system, &end_table(h));
}

extern "C" int phc_track_paths_dd(phc_homotopy *h, int64_t first, int64_t n, const phc_opts *opts, phc_cd *x_hi,
                                  phc_cd *x_lo, int8_t *cls_out, phc_path_stats *stats_out, void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (h->parameter && n > 0)
        return fail(PHC_EINVAL, "a parameter homotopy has no total-degree start system");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle is tracked by phc_track_polyhedral");
    if (n < 0 || first < 0 || first + n > h->num_paths)
        return fail(PHC_EINVAL, "path range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)h->num_paths);
    if (n == 0) return PHC_OK;
    if (!x_hi || !x_lo || !cls_out) return fail(PHC_EINVAL, "NULL output array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, s);
        if (rc) return rc;
        st = h->d_stats;
    }
    CU(cudaMemsetAsync(h->d_qhead, 0, sizeof(unsigned long long), s));
    if (h->d_tailc) CU(cudaMemsetAsync(h->d_tailc, 0, 4 * sizeof(unsigned long long), s));  // no hand-off here
    phc::TrackLaunch L{};
    L.tab = h->total.view;
    L.tab.f32 = 0;
    L.start_mode = 0;
    L.deg = h->d_deg;
    L.root_off = h->d_root_off;
    L.roots = h->d_roots;
    L.first = first;
    L.n_paths = n;
    L.paths_per_system = h->paths_per_system > 0 ? h->paths_per_system : 1;
    L.x_out = reinterpret_cast<double2 *>(x_hi);
    L.x_out2 = reinterpret_cast<double2 *>(x_lo);
    L.stats = st;
    L.qhead = h->d_qhead;
    L.o = o;
    cudaError_t e = phc::launch_track_dd(L, o.block_threads, o.max_blocks, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "double double track kernel launch: %s", cudaGetErrorString(e));
    phc::ClassifyLaunch C{};
    C.tab = end_table(h);
    C.tab.f32 = 0;
    C.n_paths = n;
    C.x = L.x_out;
    C.stats = st;
    C.cls = cls_out;
    C.o = o;
    e = phc::launch_classify(C, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "classify kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

extern "C" int phc_track_paths_qd(phc_homotopy *h, int64_t first, int64_t n, const phc_opts *opts, phc_cd *x_out,
                                  int8_t *cls_out, phc_path_stats *stats_out, void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (h->parameter && n > 0)
        return fail(PHC_EINVAL, "a parameter homotopy has no total-degree start system");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle is tracked by phc_track_polyhedral");
    if (n < 0 || first < 0 || first + n > h->num_paths)
        return fail(PHC_EINVAL, "path range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)h->num_paths);
    if (n == 0) return PHC_OK;
    if (!x_out || !cls_out) return fail(PHC_EINVAL, "NULL output array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, s);
        if (rc) return rc;
        st = h->d_stats;
    }
    CU(cudaMemsetAsync(h->d_qhead, 0, sizeof(unsigned long long), s));
    if (h->d_tailc) CU(cudaMemsetAsync(h->d_tailc, 0, 4 * sizeof(unsigned long long), s));  // no hand-off here
    phc::TrackLaunch L{};
    L.tab = h->total.view;
    L.tab.f32 = 0;
    L.start_mode = 0;
    L.deg = h->d_deg;
    L.root_off = h->d_root_off;
    L.roots = h->d_roots;
    L.first = first;
    L.n_paths = n;
    L.paths_per_system = h->paths_per_system > 0 ? h->paths_per_system : 1;
    L.x_out = reinterpret_cast<double2 *>(x_out);
    L.stats = st;
    L.qhead = h->d_qhead;
    L.o = o;
    cudaError_t e = phc::launch_track_qd(L, o.block_threads, o.max_blocks, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "quad double track kernel launch: %s", cudaGetErrorString(e));
    phc::ClassifyLaunch C{};
    C.tab = end_table(h);
    C.tab.f32 = 0;
    C.n_paths = n;
    C.x = L.x_out;  // the leading parts
    C.stats = st;
    C.cls = cls_out;
    C.o = o;
    e = phc::launch_classify(C, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "classify kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

extern "C" int phc_endgame(phc_homotopy *h, int64_t first, int64_t n, const phc_opts *opts, phc_cd *x_out,
                           int32_t *cycle_out, phc_path_stats *stats_out, void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (h->parameter && n > 0)
        return fail(PHC_EINVAL, "a parameter homotopy has no total-degree start system");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle is tracked by phc_track_polyhedral");
    if (n < 0 || first < 0 || first + n > h->num_paths)
        return fail(PHC_EINVAL, "path range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)h->num_paths);
    if (n == 0) return PHC_OK;
    if (!x_out || !cycle_out) return fail(PHC_EINVAL, "NULL output array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, s);
        if (rc) return rc;
        st = h->d_stats;
    }
    CU(cudaMemsetAsync(h->d_qhead, 0, sizeof(unsigned long long), s));
    phc::TrackLaunch L{};
    L.tab = h->total.view;
    L.tab.f32 = 0;
    L.start_mode = 0;
    L.deg = h->d_deg;
    L.root_off = h->d_root_off;
    L.roots = h->d_roots;
    L.first = first;
    L.n_paths = n;
    L.paths_per_system = h->paths_per_system > 0 ? h->paths_per_system : 1;
    L.x_out = reinterpret_cast<double2 *>(x_out);
    L.stats = st;
    L.qhead = h->d_qhead;
    L.o = o;
    cudaError_t e = phc::launch_endgame(L, cycle_out, o.block_threads, o.max_blocks, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "endgame kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

// Cascade homotopy on the handle's system E_k: every term keeps its
// coefficient (c, 0) except the terms of the last equation (hyperplane k)
// other than its slack z_k (the last unknown), which become (c, -c), i.e.
// (1-t) c.
static int ensure_cascade(phc_homotopy *h)
{
    if (h->cascade.blob) return PHC_OK;
    const int n = h->n;
    HostTerms ht;
    int64_t off = 0;
    for (int i = 0; i < n; i++) {
        for (int k = 0; k < h->tpe[i]; k++, off++) {
            const uint8_t *a = h->exps.data() + off * n;
            const phc_cd c = h->coefs[off];
            bool is_slack = a[n - 1] == 1;
            for (int j = 0; j < n - 1; j++) is_slack = is_slack && a[j] == 0;
            if (i == n - 1 && !is_slack)
                ht.add(i, a, n, make_double2(c.re, c.im), make_double2(-c.re, -c.im));
            else
                ht.add(i, a, n, make_double2(c.re, c.im), make_double2(0.0, 0.0));
        }
    }
    cudaStream_t ps = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess)
        return fail(PHC_ECUDA, "cudaStreamCreateWithFlags");
    const int rc = upload_table(ht, n, h->cascade, ps);
    cudaStreamDestroy(ps);
    return rc;
}

extern "C" int phc_cascade_stage(const phc_homotopy *hc, int k, const phc_cd *starts, int64_t n, const phc_opts *opts,
                                 phc_cd *x_out, int8_t *cls_out, uint8_t *slack_zero_out, phc_path_stats *stats_out,
                                 void *stream)
{
    phc_homotopy *h = const_cast<phc_homotopy *>(hc);
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (k < 1 || k >= h->n) return fail(PHC_EINVAL, "cascade stage k = %d outside 1..%d", k, h->n - 1);
    if (h->n_sys != 1) return fail(PHC_EUNSUPPORTED, "cascade stages need a single-system handle");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle has no cascade");
    if (n < 0) return fail(PHC_EINVAL, "n_starts < 0");
    if (n == 0) return PHC_OK;
    if (!starts || !x_out || !cls_out || !slack_zero_out) return fail(PHC_EINVAL, "NULL array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    rc = ensure_cascade(h);
    if (rc) return rc;
    rc = ensure_xfull(h, (int64_t)h->n * n, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
        st = h->d_stats;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run_track(h, h->cascade.view, 1, reinterpret_cast<const double2 *>(starts), 0, n, o, h->d_xfull, cls_out, st, s);
    if (rc) return rc;
    cudaError_t e = phc::launch_drop_last(h->d_xfull, h->n, n, reinterpret_cast<double2 *>(x_out), slack_zero_out,
                                          k > 1 ? 1 : 0, o.slack_tol, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "drop kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

// The systems of a multi-system call, grouped by number of unknowns: per
// group the descriptors, the prefix sums of the path counts and the sizes
// of the shared-memory regions of the tracker and of its tail kernel.
struct ManyGroup {
    int n = 0;
    std::vector<phc::SysDesc> descs;
    std::vector<int64_t> prefix{0};
    int wtb = 0;
    phc::TailMultiSizes tz{0, 0, 0, 0};
};

// stats_fallback(i, paths) gives the records of handle i when the caller passes none.
template <typename F>
static int many_groups(phc_homotopy *const *hs, int n_h, const phc_opts &o, phc_cd *const *x_out,
                       int8_t *const *cls_out, phc_path_stats *const *stats_out, F stats_fallback,
                       std::vector<ManyGroup> &groups)
{
    for (int i = 0; i < n_h; i++) {
        if (!hs[i]) return fail(PHC_EINVAL, "handle %d is NULL", i);
        if (hs[i]->n_sys != 1) return fail(PHC_EUNSUPPORTED, "handle %d is a batch handle", i);
        if (hs[i]->parameter) return fail(PHC_EINVAL, "handle %d is a parameter homotopy", i);
        if (hs[i]->polyhedral) return fail(PHC_EINVAL, "handle %d is a polyhedral handle", i);
        if (!x_out[i] || !cls_out[i]) return fail(PHC_EINVAL, "NULL output array of handle %d", i);
    }
    for (int n = 1; n <= PHC_MAX_VARS; n++) {
        ManyGroup g;
        g.n = n;
        for (int i = 0; i < n_h; i++) {
            phc_homotopy *h = hs[i];
            if (h->n != n || h->num_paths == 0) continue;
            phc::SysDesc d{};
            d.tab = h->total.view;
            d.tab.f32 = o.precision == PHC_PREC_FP32_INTERIOR;
            d.deg = h->d_deg;
            d.root_off = h->d_root_off;
            d.roots = h->d_roots;
            d.n_paths = h->num_paths;
            d.x_out = reinterpret_cast<double2 *>(x_out[i]);
            d.cls_out = cls_out[i];
            phc_path_stats *sp = stats_out ? stats_out[i] : nullptr;
            if (!sp) {
                const int rc = stats_fallback(i, h->num_paths, &sp);
                if (rc) return rc;
            }
            d.stats = sp;
            g.descs.push_back(d);
            g.prefix.push_back(g.prefix.back() + h->num_paths);
            const int b = (int)phc::warp_table_bytes(d.tab.n_terms, d.tab.n_ve, d.tab.f32);
            if (b > g.wtb) g.wtb = b;
            // the multi-system tail kernel's per-warp region (double precision tables)
            const int T = d.tab.n_terms, V = d.tab.n_ve, S = phc::tail_store_slots(T, V);
            g.tz.table_cap = std::max(g.tz.table_cap, phc::warp_table_bytes(T, V, false));
            g.tz.plan_cap = std::max(g.tz.plan_cap, phc::tail_plan_bytes(n, T, V));
            g.tz.group_slots = std::max(g.tz.group_slots, phc::tail_group_slots(n, S));
            g.tz.max_store = std::max(g.tz.max_store, S);
        }
        if (!g.descs.empty()) groups.push_back(std::move(g));
    }
    return PHC_OK;
}

// Device block of a group: descriptors, path counters, prefix sums, then
// (256-aligned) the 8 hand-off counters and the hand-off records.
struct ManyLayout {
    int m = 0;
    int64_t lanes = 0;
    size_t q_off = 0, pre_off = 0, hoff = 0, bytes = 0;
};

static ManyLayout many_layout(const ManyGroup &g, const phc_opts &o, phc::TrackLaunch &L)
{
    ManyLayout y;
    y.m = (int)g.descs.size();
    L = phc::TrackLaunch{};
    L.n_paths = g.prefix.back();
    L.o = o;
    L.n_multi = y.m;
    L.warp_table_bytes = g.wtb;
    const bool tail = o.tail_drain > 0.0 && phc::tail_multi_supported(g.tz);
    y.lanes = tail ? phc::multi_lanes(L, g.n, o.block_threads, o.max_blocks) : 0;
    if (y.lanes < 0) y.lanes = 0;
    y.q_off = (size_t)y.m * sizeof(phc::SysDesc);
    y.pre_off = y.q_off + (size_t)y.m * sizeof(unsigned long long);
    const size_t head = y.pre_off + (size_t)(y.m + 1) * sizeof(int64_t);
    y.hoff = (head + 255) & ~(size_t)255;
    y.bytes = y.hoff + 8 * sizeof(unsigned long long) + (size_t)y.lanes * sizeof(phc::Handoff);
    return y;
}

// Points L at a group's device block.
static void many_bind(phc::TrackLaunch &L, const ManyLayout &y, char *b, const phc_opts &o)
{
    L.multi = reinterpret_cast<const phc::SysDesc *>(b);
    L.multi_q = reinterpret_cast<unsigned long long *>(b + y.q_off);
    L.multi_prefix = reinterpret_cast<const int64_t *>(b + y.pre_off);
    unsigned long long *c = reinterpret_cast<unsigned long long *>(b + y.hoff);
    if (y.lanes > 0) {
        L.handoff_n = c;
        L.idle_n = c + 1;
        L.tail_q = c + 2;
        L.tail_units = c + 3;
        L.multi_claimed = c + 4;
        L.handoff = reinterpret_cast<phc::Handoff *>(c + 8);
        L.drain_frac = o.tail_drain;
    }
}

// Stream-ordered work of one group on stream s: counters cleared, the
// multi-system tracker and its tail kernel.  Allocates nothing.
static int many_launch(const phc::TrackLaunch &L, const ManyLayout &y, const ManyGroup &g, char *b, const phc_opts &o,
                       cudaStream_t s)
{
    CU(cudaMemsetAsync(b + y.q_off, 0, (size_t)y.m * sizeof(unsigned long long), s));
    CU(cudaMemsetAsync(b + y.hoff, 0, 8 * sizeof(unsigned long long), s));
    cudaError_t e = phc::launch_multi(L, g.n, o.block_threads, o.max_blocks, s);
    if (e == cudaSuccess && y.lanes > 0) e = phc::launch_tail_multi(L, g.n, g.tz, o.max_blocks, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "multi-system kernel launch (n = %d): %s", g.n, cudaGetErrorString(e));
    return PHC_OK;
}

// Helper streams for the groups of a call on caller stream st: each caller
// stream has helpers of its own, created with its priority, so calls on
// different streams neither wait for each other's launches nor lose their
// priority.
static int helper_streams(cudaStream_t st, size_t count, std::vector<cudaStream_t> &out)
{
    static std::mutex pool_mutex;
    static std::map<cudaStream_t, std::vector<cudaStream_t>> pools;  // nodes stay where they are
    int prio = 0;
    CU(cudaStreamGetPriority(st, &prio));
    std::lock_guard<std::mutex> lock(pool_mutex);
    std::vector<cudaStream_t> &pool = pools[st];
    while (pool.size() < count) {
        cudaStream_t ns;
        CU(cudaStreamCreateWithPriority(&ns, cudaStreamNonBlocking, prio));
        pool.push_back(ns);
    }
    out.assign(pool.begin(), pool.begin() + count);
    return PHC_OK;
}

extern "C" int phc_track_many(phc_homotopy *const *hs, int n_h, const phc_opts *opts, phc_cd *const *x_out,
                              int8_t *const *cls_out, phc_path_stats *const *stats_out, void *stream)
try {
    if (n_h < 0 || (n_h > 0 && (!hs || !x_out || !cls_out))) return fail(PHC_EINVAL, "NULL argument");
    if (n_h == 0) return PHC_OK;
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    std::vector<ManyGroup> groups;
    rc = many_groups(hs, n_h, o, x_out, cls_out, stats_out,
                     [&](int i, int64_t paths, phc_path_stats **sp) -> int {
                         const int r = ensure_stats(hs[i], paths, static_cast<cudaStream_t>(stream));
                         *sp = hs[i]->d_stats;
                         return r;
                     },
                     groups);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the launches of different sizes run side by side on helper streams
    // that fork from and join back into the caller's stream
    std::vector<cudaStream_t> helpers;
    rc = helper_streams(st, groups.size(), helpers);
    if (rc) return rc;
    cudaEvent_t fork_ev = nullptr;
    CU(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    CU(cudaEventRecord(fork_ev, st));
    std::vector<cudaEvent_t> joins;
    for (size_t gi = 0; gi < groups.size(); gi++) {
        const ManyGroup &g = groups[gi];
        cudaStream_t hs_st = helpers[gi];
        CU(cudaStreamWaitEvent(hs_st, fork_ev, 0));
        phc::TrackLaunch L;
        const ManyLayout y = many_layout(g, o, L);
        void *blob = nullptr;
        CU(cudaMallocAsync(&blob, y.bytes, hs_st));
        char *b = static_cast<char *>(blob);
        CU(cudaMemcpyAsync(b, g.descs.data(), (size_t)y.m * sizeof(phc::SysDesc), cudaMemcpyHostToDevice, hs_st));
        CU(cudaMemcpyAsync(b + y.pre_off, g.prefix.data(), (size_t)(y.m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                           hs_st));
        many_bind(L, y, b, o);
        // the host vectors must outlive the copies from pageable memory
        CU(cudaStreamSynchronize(hs_st));
        rc = many_launch(L, y, g, b, o, hs_st);
        cudaFreeAsync(blob, hs_st);
        if (rc) return rc;
        cudaEvent_t j;
        CU(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
        CU(cudaEventRecord(j, hs_st));
        joins.push_back(j);
    }
    for (cudaEvent_t j : joins) {
        CU(cudaStreamWaitEvent(st, j, 0));
        cudaEventDestroy(j);
    }
    cudaEventDestroy(fork_ev);
    return PHC_OK;
} catch (...) {
    return fail(PHC_ENOMEM, "phc_track_many: host allocation failed");
}

// ------------------------------------------------------------------ multi-system plans

struct phc_many_plan {
    phc_opts o{};
    std::vector<ManyGroup> groups;
    std::vector<ManyLayout> layouts;
    std::vector<phc::TrackLaunch> launches;
    std::vector<void *> blobs;
    std::vector<phc_path_stats *> own_stats;  // records for handles the caller gave none
    std::vector<cudaStream_t> helpers;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
};

extern "C" void phc_many_plan_destroy(phc_many_plan *p)
{
    if (!p) return;
    for (void *b : p->blobs)
        if (b) cudaFree(b);
    for (phc_path_stats *s : p->own_stats)
        if (s) cudaFree(s);
    for (cudaStream_t s : p->helpers)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : p->joins)
        if (e) cudaEventDestroy(e);
    if (p->fork) cudaEventDestroy(p->fork);
    delete p;
}

extern "C" int phc_many_plan_create(phc_homotopy *const *hs, int n_h, const phc_opts *opts, phc_cd *const *x_out,
                                    int8_t *const *cls_out, phc_path_stats *const *stats_out, void *stream,
                                    phc_many_plan **out)
try {
    if (!out) return fail(PHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_h < 1 || !hs || !x_out || !cls_out) return fail(PHC_EINVAL, "NULL argument or n_h < 1");
    phc_many_plan *p = new (std::nothrow) phc_many_plan();
    if (!p) return fail(PHC_ENOMEM, "host allocation");
    if (opts) p->o = *opts; else phc_default_opts(&p->o);
    int rc = check_opts(p->o);
    if (!rc)
        rc = many_groups(hs, n_h, p->o, x_out, cls_out, stats_out,
                         [&](int i, int64_t paths, phc_path_stats **sp) -> int {
                             (void)i;
                             *sp = nullptr;
                             if (cudaMalloc(sp, paths * sizeof(phc_path_stats)) != cudaSuccess)
                                 return fail(PHC_ENOMEM, "cudaMalloc of %lld path records", (long long)paths);
                             p->own_stats.push_back(*sp);
                             return PHC_OK;
                         },
                         p->groups);
    int prio = 0;
    if (!rc && cudaStreamGetPriority(static_cast<cudaStream_t>(stream), &prio) != cudaSuccess)
        rc = fail(PHC_ECUDA, "cudaStreamGetPriority");
    if (!rc && cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(PHC_ECUDA, "cudaEventCreate");
    for (size_t gi = 0; !rc && gi < p->groups.size(); gi++) {
        const ManyGroup &g = p->groups[gi];
        phc::TrackLaunch L;
        const ManyLayout y = many_layout(g, p->o, L);
        void *blob = nullptr;
        if (cudaMalloc(&blob, y.bytes) != cudaSuccess) {
            rc = fail(PHC_ENOMEM, "cudaMalloc of %zu bytes for the multi-system plan", y.bytes);
            break;
        }
        p->blobs.push_back(blob);
        char *b = static_cast<char *>(blob);
        if (cudaMemcpy(b, g.descs.data(), (size_t)y.m * sizeof(phc::SysDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b + y.pre_off, g.prefix.data(), (size_t)(y.m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            rc = fail(PHC_ECUDA, "upload of the multi-system descriptors");
            break;
        }
        many_bind(L, y, b, p->o);
        p->layouts.push_back(y);
        p->launches.push_back(L);
        cudaStream_t hs_st = nullptr;
        cudaEvent_t j = nullptr;
        if (cudaStreamCreateWithPriority(&hs_st, cudaStreamNonBlocking, prio) != cudaSuccess ||
            cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
            if (hs_st) cudaStreamDestroy(hs_st);
            rc = fail(PHC_ECUDA, "helper stream or event of the multi-system plan");
            break;
        }
        p->helpers.push_back(hs_st);
        p->joins.push_back(j);
    }
    if (rc) {
        phc_many_plan_destroy(p);
        return rc;
    }
    *out = p;
    return PHC_OK;
} catch (...) {
    return fail(PHC_ENOMEM, "phc_many_plan_create: host allocation failed");
}

extern "C" int phc_many_plan_run(phc_many_plan *p, void *stream)
{
    if (!p) return fail(PHC_EINVAL, "NULL plan");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CU(cudaEventRecord(p->fork, st));
    for (size_t gi = 0; gi < p->groups.size(); gi++) {
        cudaStream_t hs_st = p->helpers[gi];
        CU(cudaStreamWaitEvent(hs_st, p->fork, 0));
        const int rc = many_launch(p->launches[gi], p->layouts[gi], p->groups[gi], static_cast<char *>(p->blobs[gi]),
                                   p->o, hs_st);
        if (rc) return rc;
        CU(cudaEventRecord(p->joins[gi], hs_st));
        CU(cudaStreamWaitEvent(st, p->joins[gi], 0));
    }
    return PHC_OK;
}

static int ensure_stats2(phc_homotopy *h, int64_t n, cudaStream_t s)
{
    return grow(reinterpret_cast<void **>(&h->d_stats2), &h->stats2_cap, n, sizeof(phc_path_stats), s, "path records");
}

extern "C" int phc_track_pipeline(phc_homotopy *h, int k, int64_t first, int64_t n, const phc_opts *opts,
                                  phc_cd *x_top, int8_t *cls_top, phc_path_stats *stats_top, phc_cd *x_next,
                                  int8_t *cls_next, uint8_t *slack_zero_next, phc_path_stats *stats_next,
                                  void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (k < 1 || k >= h->n) return fail(PHC_EINVAL, "cascade stage k = %d outside 1..%d", k, h->n - 1);
    if (h->n_sys != 1) return fail(PHC_EUNSUPPORTED, "the pipeline needs a single-system handle");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle has no cascade");
    if (n < 0 || first < 0 || first + n > h->num_paths)
        return fail(PHC_EINVAL, "path range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)h->num_paths);
    if (n == 0) return PHC_OK;
    if (!x_top || !cls_top || !x_next || !cls_next || !slack_zero_next) return fail(PHC_EINVAL, "NULL output array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    rc = ensure_cascade(h);
    if (rc) return rc;
    phc_path_stats *st = stats_top, *st2 = stats_next;
    if (!st) {
        rc = ensure_stats(h, n, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
        st = h->d_stats;
    }
    if (!st2) {
        rc = ensure_stats2(h, n, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
        st2 = h->d_stats2;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CU(cudaMemsetAsync(h->d_qhead, 0, sizeof(unsigned long long), s));
    phc::TrackLaunch L{};
    L.tab = h->total.view;
    L.start_mode = 0;
    L.deg = h->d_deg;
    L.root_off = h->d_root_off;
    L.roots = h->d_roots;
    L.first = first;
    L.n_paths = n;
    L.paths_per_system = h->paths_per_system;
    L.x_out = reinterpret_cast<double2 *>(x_top);
    L.stats = st;
    L.qhead = h->d_qhead;
    L.o = o;
    L.tab2 = h->cascade.view;
    L.tab.f32 = L.tab2.f32 = o.precision == PHC_PREC_FP32_INTERIOR;
    L.cls_out = cls_top;
    L.x_out2 = reinterpret_cast<double2 *>(x_next);
    L.cls_out2 = cls_next;
    L.slack_zero2 = slack_zero_next;
    L.stats2 = st2;
    L.has_next_slack = k > 1 ? 1 : 0;
    const bool tail =
        o.tail_drain > 0.0 && phc::tail_pipe_supported(L.tab, L.tab2);
    if (tail) {
        const int64_t lanes = phc::pipe_lanes(L, o.block_threads, o.max_blocks);
        if (lanes < 1) return fail(PHC_EUNSUPPORTED, "no launch configuration for %d unknowns", L.tab.n);
        rc = ensure_handoff(h, lanes, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
        CU(cudaMemsetAsync(h->d_tailc, 0, 4 * sizeof(unsigned long long), s));
        L.handoff = h->d_handoff;
        L.handoff_n = h->d_tailc;
        L.idle_n = h->d_tailc + 1;
        L.tail_q = h->d_tailc + 2;
        L.tail_units = h->d_tailc + 3;
        L.drain_frac = o.tail_drain;
    } else if (h->d_tailc) {
        CU(cudaMemsetAsync(h->d_tailc, 0, 4 * sizeof(unsigned long long), s));
    }
    cudaError_t e = phc::launch_pipeline(L, o.block_threads, o.max_blocks, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "pipeline kernel launch: %s", cudaGetErrorString(e));
    if (tail) {
        e = phc::launch_tail_pipe(L, o.max_blocks, s);
        if (e != cudaSuccess) return fail(PHC_ECUDA, "pipelined tail kernel launch: %s", cudaGetErrorString(e));
    }
    return PHC_OK;
}

extern "C" int phc_cascade_from(const phc_homotopy *hc, int k, const phc_cd *x_prev, const int8_t *cls_prev,
                                const uint8_t *sz_prev, int64_t n, const phc_opts *opts, phc_cd *x_out,
                                int8_t *cls_out, uint8_t *slack_zero_out, phc_path_stats *stats_out, void *stream)
{
    phc_homotopy *h = const_cast<phc_homotopy *>(hc);
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (k < 1 || k >= h->n) return fail(PHC_EINVAL, "cascade stage k = %d outside 1..%d", k, h->n - 1);
    if (h->n_sys != 1) return fail(PHC_EUNSUPPORTED, "cascade stages need a single-system handle");
    if (h->polyhedral) return fail(PHC_EINVAL, "a polyhedral handle has no cascade");
    if (n < 0) return fail(PHC_EINVAL, "n < 0");
    if (n == 0) return PHC_OK;
    if (!x_prev || !cls_prev || !x_out || !cls_out || !slack_zero_out) return fail(PHC_EINVAL, "NULL array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    rc = ensure_cascade(h);
    if (rc) return rc;
    rc = ensure_xfull(h, (int64_t)h->n * n, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, static_cast<cudaStream_t>(stream));
        if (rc) return rc;
        st = h->d_stats;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run_track(h, h->cascade.view, 2, reinterpret_cast<const double2 *>(x_prev), 0, n, o, h->d_xfull, cls_out, st,
                   s, cls_prev, sz_prev);
    if (rc) return rc;
    cudaError_t e = phc::launch_drop_last(h->d_xfull, h->n, n, reinterpret_cast<double2 *>(x_out), slack_zero_out,
                                          k > 1 ? 1 : 0, o.slack_tol, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "drop kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

extern "C" int phc_membership_test(int n_eq, int n_var, const int32_t *tpe, const uint8_t *exps,
                                   const phc_cd *coefs, int k, const phc_cd *witness, int64_t m,
                                   const phc_cd *points, int64_t p, double tol, const phc_opts *opts,
                                   uint8_t *on_out, phc_cd *x_out, int8_t *cls_out, void *stream)
try {
    if (k < 1 || k >= n_var) return fail(PHC_EINVAL, "k = %d outside 1..n_var-1", k);
    if (m < 1 || p < 0) return fail(PHC_EINVAL, "need m >= 1 witness points and p >= 0 test points");
    if (p == 0) return PHC_OK;
    if (!witness || !points || !on_out) return fail(PHC_EINVAL, "NULL array");
    if (!(tol > 0.0)) return fail(PHC_EINVAL, "tol must be positive");
    if (p > 0x7fffffff) return fail(PHC_EUNSUPPORTED, "more than 2^31 - 1 test points in one call");
    int rc = validate_lists(n_eq, n_var, tpe, exps, coefs, true, nullptr);
    if (rc) return rc;
    const int n = n_var, nx = n_var - k;
    int64_t T = 0;
    for (int i = 0; i < n_eq; i++) T += tpe[i];
    // the hyperplanes are the last k equations: one constant term, linear
    // terms in x and slack terms; find the constant of each
    std::vector<int64_t> const_term(k, -1);
    {
        int64_t off = 0;
        for (int i = 0; i < n_eq; i++) {
            for (int q = 0; q < tpe[i]; q++, off++) {
                if (i < n_eq - k) continue;
                int d = 0;
                for (int j = 0; j < n; j++) d += exps[off * n + j];
                if (d > 1) return fail(PHC_EINVAL, "equation %d is not a hyperplane (term of degree %d)", i, d);
                if (d == 0) {
                    if (const_term[i - (n_eq - k)] >= 0)
                        return fail(PHC_EINVAL, "hyperplane %d has two constant terms", i);
                    const_term[i - (n_eq - k)] = off;
                }
            }
        }
        for (int j = 0; j < k; j++)
            if (const_term[j] < 0) return fail(PHC_EINVAL, "hyperplane %d has no constant term", n_eq - k + j);
    }
    for (int64_t j = 0; j < p * nx; j++)
        if (!std::isfinite(points[j].re) || !std::isfinite(points[j].im))
            return fail(PHC_EINVAL, "test point coordinate %lld is not finite", (long long)j);
    // target system of test point z: the constant of hyperplane j becomes
    // -sum_i c_ji z_i, so (z, slacks 0) satisfies every hyperplane
    std::vector<phc_cd> target((size_t)(p * T));
    for (int64_t t = 0; t < p; t++) {
        phc_cd *c = target.data() + t * T;
        std::memcpy(c, coefs, T * sizeof(phc_cd));
        const phc_cd *z = points + t * nx;
        for (int j = 0; j < k; j++) {
            const int row = n_eq - k + j;
            int64_t o2 = 0;
            for (int i = 0; i < row; i++) o2 += tpe[i];
            double re = 0.0, im = 0.0;
            for (int q = 0; q < tpe[row]; q++) {
                const int64_t term = o2 + q;
                int v = -1;
                for (int jj = 0; jj < n; jj++)
                    if (exps[term * n + jj]) v = jj;
                if (v < 0 || v >= nx) continue;
                const phc_cd a = coefs[term], zz = z[v];
                re -= a.re * zz.re - a.im * zz.im;
                im -= a.re * zz.im + a.im * zz.re;
            }
            c[const_term[j]] = {re, im};
        }
    }
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    rc = check_opts(o);
    if (rc) return rc;
    phc_homotopy *h = nullptr;
    rc = phc_make_parameter_homotopy(n_eq, n_var, tpe, exps, (int)p, coefs, target.data(), phc_cd{1.0, 0.0}, &h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t total = p * m;
    double2 *tiles = nullptr, *xo = reinterpret_cast<double2 *>(x_out), *pts = nullptr;
    int8_t *co = cls_out;
    cudaError_t e = cudaMalloc(&tiles, (size_t)total * n * sizeof(double2));
    if (e == cudaSuccess && !xo) e = cudaMalloc(&xo, (size_t)total * n * sizeof(double2));
    if (e == cudaSuccess && !co) e = cudaMalloc(&co, (size_t)total);
    if (e == cudaSuccess) e = cudaMalloc(&pts, (size_t)p * nx * sizeof(double2));
    std::vector<double2> pts_h((size_t)(p * nx));
    for (int64_t t = 0; t < p; t++)
        for (int l = 0; l < nx; l++) pts_h[(size_t)l * p + t] = make_double2(points[t * nx + l].re, points[t * nx + l].im);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pts, pts_h.data(), pts_h.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = phc::launch_tile_starts(reinterpret_cast<const double2 *>(witness), n, m, p, tiles, s);
    if (e == cudaSuccess) {
        rc = phc_track_from(h, reinterpret_cast<const phc_cd *>(tiles), total, m, &o, reinterpret_cast<phc_cd *>(xo), co,
                            nullptr, stream);
        if (!rc) e = phc::launch_match_points(xo, co, n, m, p, pts, nx, tol, on_out, s);
    }
    if (e != cudaSuccess && !rc) rc = fail(PHC_ECUDA, "membership test: %s", cudaGetErrorString(e));
    // the temporaries and the handle are released once the work is done
    const cudaError_t es = cudaStreamSynchronize(s);
    if (es != cudaSuccess && !rc) rc = fail(PHC_ECUDA, "membership test: %s", cudaGetErrorString(es));
    if (tiles) cudaFree(tiles);
    if (pts) cudaFree(pts);
    if (!x_out && xo) cudaFree(xo);
    if (!cls_out && co) cudaFree(co);
    phc_destroy_homotopy(h);
    return rc;
} catch (...) {
    return fail(PHC_ENOMEM, "phc_membership_test: host allocation failed");
}

extern "C" int phc_refine_endpoints(const phc_homotopy *hc, phc_cd *x_hi, phc_cd *x_lo, int64_t n,
                                    double cond_threshold, double cond_max, int max_iters, int8_t *cls,
                                    phc_path_stats *stats, void *stream)
{
    if (!hc) return fail(PHC_EINVAL, "NULL handle");
    if (n < 0 || max_iters < 0 || max_iters > 64) return fail(PHC_EINVAL, "n or max_iters out of range");
    if (n == 0) return PHC_OK;
    if (!x_hi || !x_lo || !cls || !stats) return fail(PHC_EINVAL, "NULL array");
    phc::RefineLaunch L{};
    L.tab = end_table(hc);
    L.n = n;
    L.x_hi = reinterpret_cast<double2 *>(x_hi);
    L.x_lo = reinterpret_cast<double2 *>(x_lo);
    L.cls = cls;
    L.stats = stats;
    L.cond_threshold = cond_threshold;
    L.cond_max = cond_max;
    L.max_iters = max_iters;
    phc_default_opts(&L.o);
    cudaError_t e = phc::launch_refine(L, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(PHC_ECUDA, "refine kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

// ------------------------------------------------------------------ embedding

// 64-bit linear congruential generator with an xorshift output (documented
// in phc.h); only used when the caller passes no constants.
struct Lcg {
    uint64_t s;
    double uniform()
    {
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        const uint64_t z = s ^ (s >> 29);
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
    phc_cd cnormal()
    {
        double u1 = uniform(), u2 = uniform();
        if (u1 < 1e-300) u1 = 1e-300;
        const double r = std::sqrt(-std::log(u1));  // |z|^2 ~ Exp(1): E|z|^2 = 1
        const double a = 2.0 * M_PI * u2;
        return {r * std::cos(a), r * std::sin(a)};
    }
};

extern "C" int phc_embed(int n_eq, int n_var, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs, int D,
                         const phc_cd *gammas, const phc_cd *hyper, uint64_t seed, phc_system_lists **out)
try {
    if (!out) return fail(PHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (D < 0) return fail(PHC_EINVAL, "top_dim = %d < 0", D);
    if (n_var + D > PHC_MAX_VARS) return fail(PHC_EINVAL, "n_var + top_dim = %d above %d", n_var + D, PHC_MAX_VARS);
    int rc = validate_lists(n_eq, n_var, tpe, exps, coefs, true, nullptr);
    if (rc) return rc;
    const int n = n_var, N = n + D;
    std::vector<phc_cd> g(gammas ? 0 : (size_t)n_eq * D), hy(hyper ? 0 : (size_t)D * (n + 1));
    if (!gammas || !hyper) {
        Lcg r{seed ^ 0x9E3779B97F4A7C15ULL};
        for (auto &v : g) v = r.cnormal();
        for (auto &v : hy) v = r.cnormal();
    }
    const phc_cd *G = gammas ? gammas : g.data();
    const phc_cd *Y = hyper ? hyper : hy.data();
    std::vector<int32_t> otpe;
    std::vector<uint8_t> oexp;
    std::vector<phc_cd> ocoef;
    int64_t off = 0;
    for (int i = 0; i < n_eq; i++) {
        for (int k = 0; k < tpe[i]; k++, off++) {
            for (int j = 0; j < n; j++) oexp.push_back(exps[off * n + j]);
            for (int j = 0; j < D; j++) oexp.push_back(0);
            ocoef.push_back(coefs[off]);
        }
        for (int k = 0; k < D; k++) {
            for (int j = 0; j < N; j++) oexp.push_back(j == n + k ? 1 : 0);
            ocoef.push_back(G[(size_t)i * D + k]);
        }
        otpe.push_back(tpe[i] + D);
    }
    for (int k = 0; k < D; k++) {
        for (int j = 0; j < N; j++) oexp.push_back(0);
        ocoef.push_back(Y[(size_t)k * (n + 1)]);
        for (int v = 0; v < n; v++) {
            for (int j = 0; j < N; j++) oexp.push_back(j == v ? 1 : 0);
            ocoef.push_back(Y[(size_t)k * (n + 1) + v + 1]);
        }
        for (int j = 0; j < N; j++) oexp.push_back(j == n + k ? 1 : 0);
        ocoef.push_back({1.0, 0.0});
        otpe.push_back(n + 2);
    }
    phc_system_lists *L = new (std::nothrow) phc_system_lists();
    if (!L) return fail(PHC_ENOMEM, "host allocation");
    L->n_eq = n_eq + D;
    L->n_var = N;
    L->n_terms = (int32_t)ocoef.size();
    L->terms_per_eq = new (std::nothrow) int32_t[otpe.size()];
    L->exps = new (std::nothrow) uint8_t[oexp.size()];
    L->coefs = new (std::nothrow) phc_cd[ocoef.size()];
    if (!L->terms_per_eq || !L->exps || !L->coefs) {
        phc_free_lists(L);
        return fail(PHC_ENOMEM, "host allocation");
    }
    std::memcpy(L->terms_per_eq, otpe.data(), otpe.size() * sizeof(int32_t));
    std::memcpy(L->exps, oexp.data(), oexp.size());
    std::memcpy(L->coefs, ocoef.data(), ocoef.size() * sizeof(phc_cd));
    *out = L;
    return PHC_OK;
} catch (...) {
    return fail(PHC_ENOMEM, "phc_embed: host allocation failed");
}

// Output lists of a host-side transformation (phc_embed, phc_square).
static int make_lists(int n_eq, int n_var, const std::vector<int32_t> &tpe, const std::vector<uint8_t> &ex,
                      const std::vector<phc_cd> &co, phc_system_lists **out)
{
    phc_system_lists *L = new (std::nothrow) phc_system_lists();
    if (!L) return fail(PHC_ENOMEM, "host allocation");
    L->n_eq = n_eq;
    L->n_var = n_var;
    L->n_terms = (int32_t)co.size();
    L->terms_per_eq = new (std::nothrow) int32_t[tpe.size()];
    L->exps = new (std::nothrow) uint8_t[ex.size() ? ex.size() : 1];
    L->coefs = new (std::nothrow) phc_cd[co.size() ? co.size() : 1];
    if (!L->terms_per_eq || !L->exps || !L->coefs) {
        phc_free_lists(L);
        return fail(PHC_ENOMEM, "host allocation");
    }
    std::memcpy(L->terms_per_eq, tpe.data(), tpe.size() * sizeof(int32_t));
    std::memcpy(L->exps, ex.data(), ex.size());
    std::memcpy(L->coefs, co.data(), co.size() * sizeof(phc_cd));
    *out = L;
    return PHC_OK;
}

extern "C" int phc_square(int n_eq, int n_var, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs,
                          const phc_cd *consts, uint64_t seed, phc_system_lists **out)
try {
    if (!out) return fail(PHC_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_lists(n_eq, n_var, tpe, exps, coefs, false, nullptr);
    if (rc) return rc;
    const int N = n_eq > n_var ? n_eq : n_var;  // unknowns and equations of the square system
    if (N > PHC_MAX_VARS) return fail(PHC_EINVAL, "the square system has %d unknowns, above %d", N, PHC_MAX_VARS);
    const int extra = N - (n_eq < n_var ? n_eq : n_var);
    const size_t n_const = n_eq < n_var ? (size_t)extra * (n_var + 1) : (size_t)n_eq * extra;
    std::vector<phc_cd> drawn(consts ? 0 : n_const);
    if (!consts) {
        Lcg r{seed ^ 0x9E3779B97F4A7C15ULL};
        for (auto &v : drawn) v = r.cnormal();
    }
    const phc_cd *C = consts ? consts : drawn.data();
    for (size_t i = 0; i < n_const; i++)
        if (!std::isfinite(C[i].re) || !std::isfinite(C[i].im)) return fail(PHC_EINVAL, "constant %zu is not finite", i);
    std::vector<int32_t> otpe;
    std::vector<uint8_t> oexp;
    std::vector<phc_cd> ocoef;
    int64_t off = 0;
    for (int i = 0; i < n_eq; i++) {
        for (int k = 0; k < tpe[i]; k++, off++) {
            for (int j = 0; j < N; j++) oexp.push_back(j < n_var ? exps[off * n_var + j] : 0);
            ocoef.push_back(coefs[off]);
        }
        int m = tpe[i];
        if (n_eq > n_var) {
            // overdetermined: every equation gains consts[i][k] s_k for the new unknowns s_k
            for (int k = 0; k < extra; k++) {
                for (int j = 0; j < N; j++) oexp.push_back(j == n_var + k ? 1 : 0);
                ocoef.push_back(C[(size_t)i * extra + k]);
            }
            m += extra;
        }
        otpe.push_back(m);
    }
    if (n_eq < n_var) {
        // underdetermined: consts[k][0] + sum_j consts[k][j+1] x_j = 0, k < n_var - n_eq
        for (int k = 0; k < extra; k++) {
            const phc_cd *h = C + (size_t)k * (n_var + 1);
            for (int j = 0; j < N; j++) oexp.push_back(0);
            ocoef.push_back(h[0]);
            for (int v = 0; v < n_var; v++) {
                for (int j = 0; j < N; j++) oexp.push_back(j == v ? 1 : 0);
                ocoef.push_back(h[v + 1]);
            }
            otpe.push_back(n_var + 1);
        }
    }
    return make_lists(N, N, otpe, oexp, ocoef, out);
} catch (...) {
    return fail(PHC_ENOMEM, "phc_square: host allocation failed");
}

extern "C" void phc_free_lists(phc_system_lists *L)
{
    if (!L) return;
    delete[] L->terms_per_eq;
    delete[] L->exps;
    delete[] L->coefs;
    delete L;
}

// ------------------------------------------------------------------ polyhedral homotopies

// Host block of the cells' data (path offsets, powers, H, U, pairs; 16-byte
// aligned parts) and the offsets of its parts.
struct PolyBlock {
    std::vector<char> host;
    size_t o_pw = 0, o_H = 0, o_U = 0, o_pr = 0;
};

static PolyBlock poly_block(const std::vector<int64_t> &path_off, const std::vector<double> &powers,
                            const std::vector<int64_t> &H, const std::vector<int64_t> &U, const int32_t *pairs,
                            size_t n_pairs)
{
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    PolyBlock B;
    B.o_pw = al(path_off.size() * sizeof(int64_t));
    B.o_H = al(B.o_pw + powers.size() * sizeof(double));
    B.o_U = al(B.o_H + H.size() * sizeof(int64_t));
    B.o_pr = al(B.o_U + U.size() * sizeof(int64_t));
    B.host.assign(al(B.o_pr + n_pairs * sizeof(int32_t)), 0);
    std::memcpy(B.host.data(), path_off.data(), path_off.size() * sizeof(int64_t));
    std::memcpy(B.host.data() + B.o_pw, powers.data(), powers.size() * sizeof(double));
    std::memcpy(B.host.data() + B.o_H, H.data(), H.size() * sizeof(int64_t));
    std::memcpy(B.host.data() + B.o_U, U.data(), U.size() * sizeof(int64_t));
    std::memcpy(B.host.data() + B.o_pr, pairs, n_pairs * sizeof(int32_t));
    return B;
}

// The terms of g with (c0, c1) = (0, c): the kernels read c from c1, and the
// classification at t = 1 sees g.
static HostTerms poly_terms(int n, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs)
{
    HostTerms ht;
    int64_t off = 0;
    for (int i = 0; i < n; i++)
        for (int k = 0; k < tpe[i]; k++, off++)
            ht.add(i, exps + off * n, n, make_double2(0.0, 0.0), make_double2(coefs[off].re, coefs[off].im));
    return ht;
}

static int make_polyhedral_homotopy(int n, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs,
                                    const int32_t *lift, const int32_t *cells, int64_t n_cells, phc_homotopy **out)
{
    if (!out) return fail(PHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_cells < 1 || !cells || !lift) return fail(PHC_EINVAL, "polyhedral homotopy: no cells or no lifting");
    if (n_cells > (1 << 30)) return fail(PHC_EUNSUPPORTED, "polyhedral homotopy: more than 2^30 cells");
    std::vector<int32_t> deg;
    int rc = validate_lists(n, n, tpe, exps, coefs, true, &deg);
    if (rc) return rc;
    int64_t T = 0;
    for (int i = 0; i < n; i++) T += tpe[i];
    const size_t nn = (size_t)n * n;
    std::vector<int64_t> path_off(n_cells + 1, 0), H(n_cells * nn), U(n_cells * nn);
    std::vector<double> powers((size_t)n_cells * T);
    for (int64_t c = 0; c < n_cells; c++) {
        const int32_t *pr = cells + (size_t)c * 2 * n;
        for (int i = 0; i < 2 * n; i++)
            if (pr[i] < 0 || pr[i] >= T) return fail(PHC_EINVAL, "cell %lld names a term outside the lists", (long long)c);
        int64_t vol = 0;
        rc = phc::cell_tracking_data(n, tpe, exps, lift, pr, &powers[(size_t)c * T], &H[c * nn], &U[c * nn], &vol);
        if (rc) return rc;
        for (int i = 0; i < 2 * n; i++)
            if (coefs[pr[i]].re == 0.0 && coefs[pr[i]].im == 0.0)
                return fail(PHC_EINVAL, "cell %lld: a term of its binomial system has a zero coefficient",
                            (long long)c);
        if (__builtin_add_overflow(path_off[c], vol, &path_off[c + 1]))
            return fail(PHC_EUNSUPPORTED, "polyhedral homotopy: more than 2^63 paths");
    }
    std::unique_ptr<phc_homotopy> own(new phc_homotopy());
    phc_homotopy *h = own.get();
    h->n = n;
    h->n_sys = 1;
    h->polyhedral = 1;
    h->n_cells = (int)n_cells;
    h->tpe.assign(tpe, tpe + n);
    h->exps.assign(exps, exps + T * n);
    h->coefs.assign(coefs, coefs + T);
    h->deg = deg;
    h->num_paths = path_off[n_cells];
    h->paths_per_system = h->num_paths;
    cudaGetDevice(&h->device);
    const PolyBlock B = poly_block(path_off, powers, H, U, cells, (size_t)n_cells * 2 * n);
    const HostTerms terms = poly_terms(n, tpe, exps, coefs);
    cudaStream_t ps = nullptr;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess)
        return fail(PHC_ECUDA, "cudaStreamCreateWithFlags");
    own.release();  // from here phc_destroy_homotopy frees h and its device memory
    rc = upload_table(terms, n, h->total, ps);
    if (!rc && cudaMalloc(&h->d_poly, B.host.size()) != cudaSuccess) rc = fail(PHC_ENOMEM, "cudaMalloc of the cell data");
    if (!rc && (cudaMemcpyAsync(h->d_poly, B.host.data(), B.host.size(), cudaMemcpyHostToDevice, ps) != cudaSuccess ||
                cudaStreamSynchronize(ps) != cudaSuccess))
        rc = fail(PHC_ECUDA, "upload of the cell data");
    cudaStreamDestroy(ps);
    if (!rc && cudaMalloc(&h->d_qhead, sizeof(unsigned long long)) != cudaSuccess)
        rc = fail(PHC_ENOMEM, "cudaMalloc of the path counter");
    if (rc) {
        phc_destroy_homotopy(h);
        return rc;
    }
    char *b = static_cast<char *>(h->d_poly);
    h->d_path_off = reinterpret_cast<const int64_t *>(b);
    h->d_powers = reinterpret_cast<const double *>(b + B.o_pw);
    h->d_H = reinterpret_cast<const int64_t *>(b + B.o_H);
    h->d_U = reinterpret_cast<const int64_t *>(b + B.o_U);
    h->d_pairs = reinterpret_cast<const int32_t *>(b + B.o_pr);
    *out = h;
    return PHC_OK;
}

extern "C" int phc_make_polyhedral_homotopy(int n, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs,
                                            const int32_t *lift, const int32_t *cells, int64_t n_cells,
                                            phc_homotopy **out)
{
    try {
        return make_polyhedral_homotopy(n, tpe, exps, coefs, lift, cells, n_cells, out);
    } catch (...) {
        return fail(PHC_ENOMEM, "phc_make_polyhedral_homotopy: host allocation failed");
    }
}

static phc::PolyLaunch poly_launch(const DevTables &tab, int n_cells, const char *block, const PolyBlock &B,
                                   int64_t first, int64_t n, double2 *x_out)
{
    phc::PolyLaunch L{};
    L.tab = tab;
    L.tab.f32 = 0;
    L.n_cells = n_cells;
    L.path_off = reinterpret_cast<const int64_t *>(block);
    L.powers = reinterpret_cast<const double *>(block + B.o_pw);
    L.H = reinterpret_cast<const int64_t *>(block + B.o_H);
    L.U = reinterpret_cast<const int64_t *>(block + B.o_U);
    L.pairs = reinterpret_cast<const int32_t *>(block + B.o_pr);
    L.first = first;
    L.n_paths = n;
    L.x_out = x_out;
    return L;
}

static phc::PolyLaunch handle_poly_launch(const phc_homotopy *h, int64_t first, int64_t n, double2 *x_out)
{
    phc::PolyLaunch L{};
    L.tab = h->total.view;
    L.tab.f32 = 0;
    L.n_cells = h->n_cells;
    L.path_off = h->d_path_off;
    L.powers = h->d_powers;
    L.H = h->d_H;
    L.U = h->d_U;
    L.pairs = h->d_pairs;
    L.first = first;
    L.n_paths = n;
    L.x_out = x_out;
    return L;
}

extern "C" int phc_polyhedral_starts(const phc_homotopy *h, int64_t first, int64_t n, phc_cd *x_out, void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (!h->polyhedral) return fail(PHC_EINVAL, "not a polyhedral handle");
    if (n < 0 || first < 0 || first + n > h->num_paths)
        return fail(PHC_EINVAL, "path range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)h->num_paths);
    if (n == 0) return PHC_OK;
    if (!x_out) return fail(PHC_EINVAL, "NULL output array");
    const phc::PolyLaunch L = handle_poly_launch(h, first, n, reinterpret_cast<double2 *>(x_out));
    cudaError_t e = phc::launch_poly_starts(L, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(PHC_ECUDA, "start solution kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

static int classify_poly(const DevTables &tab, int64_t n, const double2 *x, int64_t x_ld, phc_path_stats *st,
                         int8_t *cls, const phc_opts &o, cudaStream_t s)
{
    phc::ClassifyLaunch C{};
    C.tab = tab;
    C.tab.f32 = 0;
    C.n_paths = n;
    C.x = x;
    C.x_ld = x_ld;
    C.stats = st;
    C.cls = cls;
    C.o = o;
    cudaError_t e = phc::launch_classify(C, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "classify kernel launch: %s", cudaGetErrorString(e));
    return PHC_OK;
}

extern "C" int phc_track_polyhedral(phc_homotopy *h, int64_t first, int64_t n, const phc_opts *opts, phc_cd *x_out,
                                    int8_t *cls_out, phc_path_stats *stats_out, void *stream)
{
    if (!h) return fail(PHC_EINVAL, "NULL handle");
    if (!h->polyhedral) return fail(PHC_EINVAL, "not a polyhedral handle");
    if (n < 0 || first < 0 || first + n > h->num_paths)
        return fail(PHC_EINVAL, "path range [%lld, %lld) outside [0, %lld)", (long long)first,
                    (long long)(first + n), (long long)h->num_paths);
    if (n == 0) return PHC_OK;
    if (!x_out || !cls_out) return fail(PHC_EINVAL, "NULL output array");
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    int rc = check_opts(o);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    phc_path_stats *st = stats_out;
    if (!st) {
        rc = ensure_stats(h, n, s);
        if (rc) return rc;
        st = h->d_stats;
    }
    CU(cudaMemsetAsync(h->d_qhead, 0, sizeof(unsigned long long), s));
    if (h->d_tailc) CU(cudaMemsetAsync(h->d_tailc, 0, 4 * sizeof(unsigned long long), s));  // no hand-off here
    phc::PolyLaunch L = handle_poly_launch(h, first, n, reinterpret_cast<double2 *>(x_out));
    L.stats = st;
    L.qhead = h->d_qhead;
    L.o = o;
    cudaError_t e = phc::launch_track_poly(L, o.block_threads, o.max_blocks, s);
    if (e != cudaSuccess) return fail(PHC_ECUDA, "polyhedral track kernel launch: %s", cudaGetErrorString(e));
    return classify_poly(h->total.view, n, L.x_out, 0, st, cls_out, o, s);
}

// The two-stage pipeline of Section 2.2 (Figure 2): this thread makes the
// cells one after the other (the first stage) while the GPU tracks the paths
// of the cells made so far (the second stage).  Cells are gathered into
// batches of growing size (the first small, so that tracking starts early);
// each batch is uploaded and launched on one of a few helper streams, so
// batches overlap on the GPU, and its cell data are freed in stream order.
static int solve_polyhedral(int n, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs, const int32_t *lift,
                            const phc_opts *opts, int64_t max_paths, phc_cd *x_out, int8_t *cls_out,
                            phc_path_stats *stats_out, int64_t *n_paths_out, int64_t *n_cells_out, void *stream)
{
    if (!n_paths_out) return fail(PHC_EINVAL, "n_paths_out is NULL");
    *n_paths_out = 0;
    if (n_cells_out) *n_cells_out = 0;
    if (max_paths < 0) return fail(PHC_EINVAL, "max_paths < 0");
    if (max_paths > 0 && (!x_out || !cls_out)) return fail(PHC_EINVAL, "NULL output array");
    if (!lift) return fail(PHC_EINVAL, "NULL lifting");
    std::vector<int32_t> deg;
    int rc = validate_lists(n, n, tpe, exps, coefs, true, &deg);
    if (rc) return rc;
    phc_opts o;
    if (opts) o = *opts; else phc_default_opts(&o);
    rc = check_opts(o);
    if (rc) return rc;
    int64_t T = 0;
    for (int i = 0; i < n; i++) T += tpe[i];
    const size_t nn = (size_t)n * n;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    constexpr int K = 8;  // helper streams
    DeviceTable tab;
    cudaStream_t hs[K] = {};
    cudaEvent_t ev[K + 1] = {};
    unsigned long long *counters = nullptr;
    phc_path_stats *st = stats_out;
    bool own_stats = false;
    auto cleanup = [&]() {
        free_table(tab);
        if (counters) cudaFree(counters);
        if (own_stats && st) cudaFree(st);
        for (int k = 0; k < K; k++)
            if (hs[k]) cudaStreamDestroy(hs[k]);
        for (int k = 0; k <= K; k++)
            if (ev[k]) cudaEventDestroy(ev[k]);
    };
    {
        cudaStream_t ps = nullptr;
        if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess)
            return fail(PHC_ECUDA, "cudaStreamCreateWithFlags");
        rc = upload_table(poly_terms(n, tpe, exps, coefs), n, tab, ps);
        cudaStreamDestroy(ps);
        if (rc) return rc;
    }
    int prio = 0;
    if (cudaStreamGetPriority(s, &prio) != cudaSuccess) prio = 0;
    for (int k = 0; k < K && !rc; k++)
        if (cudaStreamCreateWithPriority(&hs[k], cudaStreamNonBlocking, prio) != cudaSuccess)
            rc = fail(PHC_ECUDA, "cudaStreamCreateWithPriority");
    for (int k = 0; k <= K && !rc; k++)
        if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess)
            rc = fail(PHC_ECUDA, "cudaEventCreateWithFlags");
    if (!rc && cudaMalloc(&counters, K * sizeof(unsigned long long)) != cudaSuccess)
        rc = fail(PHC_ENOMEM, "cudaMalloc of the path counters");
    if (!rc && !st && max_paths > 0) {
        if (cudaMalloc(&st, (size_t)max_paths * sizeof(phc_path_stats)) != cudaSuccess)
            rc = fail(PHC_ENOMEM, "cudaMalloc of the path records");
        own_stats = true;
    }
    // fork: the helper streams start after the work already on the caller's stream
    if (!rc && cudaEventRecord(ev[K], s) != cudaSuccess) rc = fail(PHC_ECUDA, "cudaEventRecord");
    for (int k = 0; k < K && !rc; k++)
        if (cudaStreamWaitEvent(hs[k], ev[K], 0) != cudaSuccess) rc = fail(PHC_ECUDA, "cudaStreamWaitEvent");
    if (rc) {
        cudaStreamSynchronize(s);
        cleanup();
        return rc;
    }

    int64_t launched = 0, mv = 0, cells = 0, limit = 64;
    bool overflow = false;
    // Host allocations below may throw: the GPU work already queued is still
    // joined and synchronized before the resources go.
    try {
        std::vector<int64_t> b_off(1, 0), b_H, b_U;
        std::vector<double> b_pw;
        std::vector<int32_t> b_pairs;
        int next = 0;
        auto flush = [&]() -> int {
            const int64_t paths = b_off.back();
            const int64_t nc = (int64_t)b_off.size() - 1;
            if (nc == 0) return PHC_OK;
            if (launched + paths > max_paths) overflow = true;
            if (!overflow) {
                const PolyBlock B = poly_block(b_off, b_pw, b_H, b_U, b_pairs.data(), b_pairs.size());
                cudaStream_t hk = hs[next];
                void *blk = nullptr;
                CU(cudaMallocAsync(&blk, B.host.size(), hk));
                // pageable source: staged before the call returns, so B may go
                CU(cudaMemcpyAsync(blk, B.host.data(), B.host.size(), cudaMemcpyHostToDevice, hk));
                phc::PolyLaunch L = poly_launch(tab.view, (int)nc, static_cast<const char *>(blk), B, 0, paths,
                                                reinterpret_cast<double2 *>(x_out) + launched);
                L.x_ld = max_paths;
                L.stats = st + launched;
                L.qhead = counters + next;
                L.o = o;
                CU(cudaMemsetAsync(counters + next, 0, sizeof(unsigned long long), hk));
                cudaError_t e = phc::launch_track_poly(L, o.block_threads, o.max_blocks, hk);
                if (e != cudaSuccess) return fail(PHC_ECUDA, "polyhedral track kernel launch: %s", cudaGetErrorString(e));
                CU(cudaFreeAsync(blk, hk));
                launched += paths;
                next = (next + 1) % K;
            }
            b_off.assign(1, 0);
            b_H.clear();
            b_U.clear();
            b_pw.clear();
            b_pairs.clear();
            if (limit < 16384) limit *= 2;
            return PHC_OK;
        };
        rc = phc::enumerate_mixed_cells(n, tpe, exps, lift, [&](const int32_t *pairs, int64_t) -> int {
            const size_t c = b_off.size() - 1;
            b_H.resize((c + 1) * nn);
            b_U.resize((c + 1) * nn);
            b_pw.resize((c + 1) * (size_t)T);
            int64_t vol = 0;
            const int r = phc::cell_tracking_data(n, tpe, exps, lift, pairs, &b_pw[c * T], &b_H[c * nn], &b_U[c * nn], &vol);
            if (r) return r;
            for (int i = 0; i < 2 * n; i++)
                if (coefs[pairs[i]].re == 0.0 && coefs[pairs[i]].im == 0.0)
                    return fail(PHC_EINVAL, "a cell's binomial system has a zero coefficient");
            b_pairs.insert(b_pairs.end(), pairs, pairs + 2 * n);
            b_off.push_back(b_off.back() + vol);
            cells++;
            if (__builtin_add_overflow(mv, vol, &mv)) return fail(PHC_EUNSUPPORTED, "mixed volume above 2^63");
            return b_off.back() >= limit ? flush() : PHC_OK;
        });
        if (!rc) rc = flush();
    } catch (...) {
        rc = fail(PHC_ENOMEM, "polyhedral pipeline: host allocation failed");
    }
    // join, then classify every path at t = 1 on the caller's stream
    for (int k = 0; k < K; k++)
        if ((cudaEventRecord(ev[k], hs[k]) != cudaSuccess || cudaStreamWaitEvent(s, ev[k], 0) != cudaSuccess) && !rc)
            rc = fail(PHC_ECUDA, "joining the helper streams");
    if (!rc && !overflow && launched > 0)
        rc = classify_poly(tab.view, launched, reinterpret_cast<const double2 *>(x_out), max_paths, st, cls_out, o, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (!rc && e != cudaSuccess) rc = fail(PHC_ECUDA, "polyhedral pipeline: %s", cudaGetErrorString(e));
    cleanup();
    if (rc) return rc;
    *n_paths_out = mv;
    if (n_cells_out) *n_cells_out = cells;
    if (overflow)
        return fail(PHC_EINVAL, "the mixed volume %lld exceeds max_paths %lld", (long long)mv, (long long)max_paths);
    return PHC_OK;
}

extern "C" int phc_solve_polyhedral(int n, const int32_t *tpe, const uint8_t *exps, const phc_cd *coefs,
                                    const int32_t *lift, const phc_opts *opts, int64_t max_paths, phc_cd *x_out,
                                    int8_t *cls_out, phc_path_stats *stats_out, int64_t *n_paths_out,
                                    int64_t *n_cells_out, void *stream)
{
    try {
        return solve_polyhedral(n, tpe, exps, coefs, lift, opts, max_paths, x_out, cls_out, stats_out, n_paths_out,
                                n_cells_out, stream);
    } catch (...) {
        return fail(PHC_ENOMEM, "phc_solve_polyhedral: host allocation failed");
    }
}

// ------------------------------------------------------------------ internal accessors (noalloc.cu)

namespace phc {

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

int check_options(const phc_opts &o) { return check_opts(o); }

int handle_num_paths(const phc_homotopy *h, int64_t *out)
{
    *out = h->num_paths;
    return PHC_OK;
}

// Device view of the handle's total-degree homotopy and start tables, set
// up for the options' arithmetic as run_track sets it up (the single
// precision copies staged only for FP32_INTERIOR).
int handle_track_view(phc_homotopy *h, const phc_opts &o, TrackLaunch *L)
{
    if (h->parameter || h->polyhedral) return fail(PHC_EINVAL, "the handle has no total-degree start system");
    L->tab = h->total.view;
    L->tab.f32 = o.precision == PHC_PREC_FP32_INTERIOR;
    L->deg = h->d_deg;
    L->root_off = h->d_root_off;
    L->roots = h->d_roots;
    L->paths_per_system = h->paths_per_system;
    return PHC_OK;
}

// The handle's hand-off counters (NULL until a call used the hand-off):
// phc_tail_paths reads them.
unsigned long long *handle_tail_counters(phc_homotopy *h) { return h->d_tailc; }

}  // namespace phc
