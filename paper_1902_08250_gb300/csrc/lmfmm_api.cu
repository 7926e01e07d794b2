// lmfmm_api.cu -- the C ABI declared in include/lmfmm.h: argument checks,
// handle management and error reporting around the setup and apply code.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "internal.h"

static thread_local char g_err[512] = "";

void lm_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" const char *lm_last_error(void) { return g_err; }

extern "C" const char *lm_status_string(lm_status s)
{
    switch (s) {
    case LM_OK: return "ok";
    case LM_EINVAL: return "invalid argument";
    case LM_ENOMEM: return "out of memory";
    case LM_ECUDA: return "CUDA error";
    case LM_ETIMEOUT: return "device wait timed out";
    case LM_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

extern "C" lm_status lm_options_default(lm_options *o)
{
    if (!o) {
        lm_set_error("options_default: NULL pointer");
        return LM_EINVAL;
    }
    o->p = 20;
    o->depth = -1;
    o->leaf_target = 48;
    o->precision = LM_FP64;
    o->max_nvec = 16;
    o->seg_order = 16;
    o->tail_order = 0;
    o->tail_rays = 9;
    return LM_OK;
}

static bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

extern "C" lm_status lm_create_medium(double k1, double k2, double k3, double d, const lm_options *opt,
                                      lm_medium *out)
{
    if (!out) {
        lm_set_error("create_medium: out is NULL");
        return LM_EINVAL;
    }
    *out = nullptr;
    if (!finite_pos(k1) || !finite_pos(k2) || !finite_pos(k3) || !finite_pos(d)) {
        lm_set_error("create_medium: k1, k2, k3 and d must be finite and > 0");
        return LM_EINVAL;
    }
    lm_options o;
    lm_options_default(&o);
    if (opt) o = *opt;
    if (o.p == 0) o.p = 20;
    if (o.leaf_target <= 0) o.leaf_target = 48;
    if (o.max_nvec <= 0) o.max_nvec = 16;
    if (o.seg_order <= 0) o.seg_order = 16;
    if (o.tail_rays <= 0) o.tail_rays = 9;
    if (o.tail_order <= 0) o.tail_order = o.precision == LM_MIXED ? 24 : 64;
    if (o.p < 1 || o.p > LM_MAXP) {
        lm_set_error("create_medium: p must be in 1..%d", LM_MAXP);
        return LM_EINVAL;
    }
    if (o.depth > 14 || o.depth < -1) {
        lm_set_error("create_medium: depth must be -1 or 0..14");
        return LM_EINVAL;
    }
    if (o.precision != LM_FP64 && o.precision != LM_MIXED) {
        lm_set_error("create_medium: unknown precision %d", o.precision);
        return LM_EINVAL;
    }
    if (o.seg_order > 64 || o.tail_order > 256 || o.tail_rays > 64) {
        lm_set_error("create_medium: quadrature orders out of range");
        return LM_EINVAL;
    }
    lm_medium_s *m = new (std::nothrow) lm_medium_s();
    if (!m) {
        lm_set_error("create_medium: host allocation failed");
        return LM_ENOMEM;
    }
    m->k1 = k1;
    m->k2 = k2;
    m->k3 = k3;
    m->d = d;
    m->opt = o;
    *out = m;
    return LM_OK;
}

extern "C" void lm_destroy_medium(lm_medium m) { delete m; }

extern "C" void lm_destroy_tree(lm_tree t)
{
    if (!t) return;
    lm_free_tree_device(t);
    delete t;
}

extern "C" lm_status lm_build_tree(lm_medium m, const double *x, const double *y, int64_t n, void *stream,
                                   lm_tree *out)
{
    if (!out) {
        lm_set_error("build_tree: out is NULL");
        return LM_EINVAL;
    }
    *out = nullptr;
    if (!m || !x || !y || n < 1) {
        lm_set_error("build_tree: NULL medium or coordinates, or n < 1");
        return LM_EINVAL;
    }
    if (n > INT32_MAX) {
        lm_set_error("build_tree: n beyond 2^31 - 1 is not supported");
        return LM_ENOTSUP;
    }
    cudaStream_t st = (cudaStream_t)stream;
    lm_tree_s *t = new (std::nothrow) lm_tree_s();
    if (!t) {
        lm_set_error("build_tree: host allocation failed");
        return LM_ENOMEM;
    }
    t->med = *m;
    t->n = n;
    t->p = m->opt.p;
    t->np = 2 * t->p + 1;
    t->precision = m->opt.precision;
    t->max_nvec = m->opt.max_nvec;
    lm_status s = lm_setup_tree(t, x, y, st);
    if (s == LM_OK) s = lm_setup_tables(t, st);
    if (s != LM_OK) {
        cudaStreamSynchronize(st);
        lm_destroy_tree(t);
        return s;
    }
    *out = t;
    return LM_OK;
}

static lm_status check_apply(lm_tree t, const void *q, int nvec, void *u)
{
    if (!t || !q || !u || nvec < 1) {
        lm_set_error("apply: NULL tree or buffer, or nvec < 1");
        return LM_EINVAL;
    }
    const char *a = (const char *)q, *b = (const char *)u;
    size_t bytes = (size_t)nvec * t->n * sizeof(zd);
    if (a < b + bytes && b < a + bytes) {
        lm_set_error("apply: q and u overlap");
        return LM_EINVAL;
    }
    return LM_OK;
}

extern "C" lm_status lm_apply(lm_tree t, const void *q, int nvec, void *u, void *stream)
{
    lm_status s = check_apply(t, q, nvec, u);
    if (s != LM_OK) return s;
    return lm_run_apply(t, (const zd *)q, nvec, (zd *)u, false, (cudaStream_t)stream);
}

extern "C" lm_status lm_apply_adjoint(lm_tree t, const void *v, int nvec, void *w, void *stream)
{
    lm_status s = check_apply(t, v, nvec, w);
    if (s != LM_OK) return s;
    return lm_run_apply(t, (const zd *)v, nvec, (zd *)w, true, (cudaStream_t)stream);
}

extern "C" lm_status lm_get_tree_info(lm_tree t, lm_tree_info *info)
{
    if (!t || !info) {
        lm_set_error("get_tree_info: NULL argument");
        return LM_EINVAL;
    }
    info->n = t->n;
    info->R = t->R;
    info->depth = t->L;
    info->p = t->p;
    info->x_origin = t->x0;
    info->nleaf = t->nleaf;
    info->precision = t->precision;
    info->max_nvec = t->max_nvec;
    info->device_bytes = t->bytes;
    return LM_OK;
}

extern "C" lm_status lm_tree_export(lm_tree t, int64_t *perm, int64_t *leaf_start, void *stream)
{
    if (!t) {
        lm_set_error("tree_export: NULL tree");
        return LM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (perm) LM_CUDA(cudaMemcpyAsync(perm, t->perm, t->n * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (leaf_start)
        LM_CUDA(cudaMemcpyAsync(leaf_start, t->leaf_start, (t->nleaf + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    return LM_OK;
}

extern "C" lm_status lm_list_export(lm_tree t, int which, int level, int64_t *out, int64_t cap,
                                    int64_t *count, void *stream)
{
    if (!t || !count || (which != 0 && which != 1) || cap < 0 || (cap > 0 && !out)) {
        lm_set_error("list_export: bad argument");
        return LM_EINVAL;
    }
    std::vector<int64_t> rows;
    lm_status s = lm_list_to_host(t, which, level, rows, (cudaStream_t)stream);
    if (s != LM_OK) return s;
    int64_t ne = (int64_t)rows.size() / 3;
    *count = ne;
    if (cap > 0) memcpy(out, rows.data(), std::min(cap, ne) * 3 * sizeof(int64_t));
    return LM_OK;
}

extern "C" lm_status lm_m2l_table_export(lm_tree t, int level, int term, int dc, int dr, double *out,
                                         void *stream)
{
    if (!t || !out || level < 0 || level > t->L) {
        lm_set_error("m2l_table_export: bad argument");
        return LM_EINVAL;
    }
    Level &lv = t->lev[level];
    int slot = -1;
    for (size_t i = 0; i < lv.cls_term.size(); ++i)
        if (lv.cls_term[i] == term && lv.cls_dc[i] == dc && lv.cls_dr[i] == dr) slot = (int)i;
    if (slot < 0) {
        lm_set_error("m2l_table_export: class (level %d, term %d, dc %d, dr %d) is in no list", level,
                     term, dc, dr);
        return LM_EINVAL;
    }
    const int P = t->p, np = 2 * P + 1;
    std::vector<zd> tab(np * np);
    std::vector<double> sc(P + 1);
    cudaStream_t st = (cudaStream_t)stream;
    LM_CUDA(cudaMemcpyAsync(tab.data(), lv.tab + (int64_t)slot * np * np, np * np * sizeof(zd),
                            cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(sc.data(), lv.scale, (P + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    // undo the scaling S(p) S(q)
    for (int p = -P; p <= P; ++p)
        for (int q = -P; q <= P; ++q) {
            double s = sc[abs(p)] * sc[abs(q)];
            zd v = tab[(p + P) * np + (q + P)];
            out[2 * ((p + P) * np + (q + P))] = v.re / s;
            out[2 * ((p + P) * np + (q + P)) + 1] = v.im / s;
        }
    return LM_OK;
}
