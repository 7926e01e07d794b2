// lmfmm_api.cu -- the C ABI declared in include/lmfmm.h: argument checks,
// handle management and error reporting around the setup and apply code.
#include <math.h>
#include <mutex>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "internal.h"

static thread_local char g_err[512] = "";
void lm_profile_apply_start(lm_tree_s *t);
void lm_profile_apply_stop(lm_tree_s *t);

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
    o->seg_order = 0;
    o->tail_order = 0;
    o->tail_rays = 9;
    o->tensor_m2l = 1;
    o->kernel = LM_KERNEL_G;
    o->autotune = 0;
    o->top_bc = LM_BC_TRANSMISSION;
    o->bottom_bc = LM_BC_TRANSMISSION;
    o->top_alpha = 0.0;
    o->bottom_alpha = 0.0;
    o->adaptive = 0;
    o->m2l_fp64 = 0;
    o->tensor_leaf = 1;
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
    if (o.seg_order <= 0) o.seg_order = o.precision == LM_MIXED ? 10 : 16;
    if (o.tail_rays <= 0) o.tail_rays = 9;
    if (o.tail_order <= 0) {
        // an impedance wall's reflection tends to 1 like 1/lambda: its tail converges more slowly
        const bool imp = o.top_bc == LM_BC_IMPEDANCE || o.bottom_bc == LM_BC_IMPEDANCE;
        o.tail_order = o.precision == LM_MIXED ? 24 : (imp ? 192 : 48);
    }
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
    if (o.top_bc < LM_BC_TRANSMISSION || o.top_bc > LM_BC_IMPEDANCE || o.bottom_bc < LM_BC_TRANSMISSION ||
        o.bottom_bc > LM_BC_IMPEDANCE || !isfinite(o.top_alpha) || !isfinite(o.bottom_alpha)) {
        lm_set_error("create_medium: unknown boundary kind or non-finite impedance alpha");
        return LM_EINVAL;
    }
    if (o.kernel != LM_KERNEL_G && o.kernel != LM_KERNEL_DG_DD) {
        lm_set_error("create_medium: unknown kernel %d", o.kernel);
        return LM_EINVAL;
    }
    if (o.m2l_fp64 != 0 && o.m2l_fp64 != 1) {
        lm_set_error("create_medium: m2l_fp64 must be 0 or 1");
        return LM_EINVAL;
    }
    if (o.adaptive != 0 && o.adaptive != 1) {
        lm_set_error("create_medium: adaptive must be 0 or 1");
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
    for (cudaEvent_t e : t->prof_ev) cudaEventDestroy(e);
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
    t->m2l_df = t->precision == LM_FP64 && m->opt.m2l_fp64 == 0;
    lm_status s;
    if (m->opt.adaptive) {
        s = lm_setup_adaptive(t, x, y, st);
    } else {
        s = lm_setup_tree(t, x, y, st);
        if (s == LM_OK) s = lm_setup_tables(t, st);
    }
    if (s == LM_OK && t->precision == LM_MIXED && !t->adaptive && m->opt.autotune)
        s = lm_autotune_mixed(t, st, nullptr, nullptr);
    if (s != LM_OK) {
        cudaStreamSynchronize(st);
        lm_destroy_tree(t);
        return s;
    }
    *out = t;
    return LM_OK;
}

static lm_status check_apply(lm_tree t, const void *q, int nvec, void *u, size_t esize = sizeof(zd))
{
    if (!t || !q || !u || nvec < 1) {
        lm_set_error("apply: NULL tree or buffer, or nvec < 1");
        return LM_EINVAL;
    }
    const char *a = (const char *)q, *b = (const char *)u;
    size_t bytes = (size_t)nvec * t->n * esize;
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
    lm_profile_apply_start(t);
    s = lm_run_apply(t, (const zd *)q, nvec, (zd *)u, false, (cudaStream_t)stream);
    lm_profile_apply_stop(t);
    return s;
}

extern "C" lm_status lm_apply_adjoint(lm_tree t, const void *v, int nvec, void *w, void *stream)
{
    lm_status s = check_apply(t, v, nvec, w);
    if (s != LM_OK) return s;
    lm_profile_apply_start(t);
    s = lm_run_apply(t, (const zd *)v, nvec, (zd *)w, true, (cudaStream_t)stream);
    lm_profile_apply_stop(t);
    return s;
}

extern "C" lm_status lm_autotune(lm_tree t, void *stream, int *choice, float *ms)
{
    if (!t) {
        lm_set_error("autotune: NULL tree");
        return LM_EINVAL;
    }
    if (t->precision != LM_MIXED || t->adaptive) { // no tile shapes to choose: FP64, or the adaptive tree's list M2L
        for (int l = 0; l <= t->L; ++l) {
            if (choice) choice[l] = -1;
            if (ms) ms[l] = 0.f;
        }
        return LM_OK;
    }
    return lm_autotune_mixed(t, (cudaStream_t)stream, choice, ms);
}

static lm_status apply_c64(lm_tree t, const void *q, int nvec, void *u, bool adjoint, void *stream)
{
    lm_status s = check_apply(t, q, nvec, u, sizeof(zf));
    if (s != LM_OK) return s;
    if (t->precision != LM_MIXED) {
        lm_set_error("apply_c64: complex64 buffers need an LM_MIXED tree");
        return LM_EINVAL;
    }
    lm_profile_apply_start(t);
    s = lm_run_apply_mixed(t, q, nvec, u, adjoint, true, (cudaStream_t)stream);
    lm_profile_apply_stop(t);
    return s;
}

extern "C" lm_status lm_apply_c64(lm_tree t, const void *q, int nvec, void *u, void *stream)
{
    return apply_c64(t, q, nvec, u, false, stream);
}

extern "C" lm_status lm_apply_adjoint_c64(lm_tree t, const void *v, int nvec, void *w, void *stream)
{
    return apply_c64(t, v, nvec, w, true, stream);
}

extern "C" lm_status lm_apply_grad(lm_tree t, const void *q, int nvec, void *u, void *ux, void *uy,
                                   void *stream)
{
    lm_status s = check_apply(t, q, nvec, ux);
    if (s != LM_OK) return s;
    s = check_apply(t, q, nvec, uy);
    if (s != LM_OK) return s;
    if (u) {
        s = check_apply(t, q, nvec, u);
        if (s != LM_OK) return s;
    }
    if (t->precision != LM_FP64) {
        lm_set_error("apply_grad: FP64 trees only");
        return LM_ENOTSUP;
    }
    lm_profile_apply_start(t);
    s = lm_run_apply_grad(t, (const zd *)q, nvec, (zd *)u, (zd *)ux, (zd *)uy, (cudaStream_t)stream);
    lm_profile_apply_stop(t);
    return s;
}

extern "C" lm_status lm_set_poll_limit(lm_tree t, int limit)
{
    if (!t) {
        lm_set_error("set_poll_limit: NULL tree");
        return LM_EINVAL;
    }
    t->tt_poll_limit = limit < 0 ? -1 : limit;
    return LM_OK;
}

extern "C" lm_status lm_sync_status(lm_tree t, void *stream)
{
    if (!t) {
        lm_set_error("sync_status: NULL tree");
        return LM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int f = 0;
    LM_CUDA(cudaMemcpyAsync(&f, t->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    if (f) {
        LM_CUDA(cudaMemsetAsync(t->dflag + 1, 0, sizeof(int), st));
        LM_CUDA(cudaStreamSynchronize(st));
        lm_set_error("a bounded wait in the tensor-core M2L gave up; the apply result is invalid");
        return LM_ETIMEOUT;
    }
    return LM_OK;
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
    info->adaptive = t->adaptive ? 1 : 0;
    info->tensor_leaf = (t->lf_ready && lm_mixed_tiles(t, LM_MAXV)) ? 1 : 0;
    if (t->adaptive) {
        info->nbox = t->at.nbox;
    } else {
        int64_t nb = 0;
        for (int l = 0; l <= t->L; ++l) nb += ((int64_t)t->R << l) << l;
        info->nbox = nb;
    }
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
        LM_CUDA(cudaMemcpyAsync(leaf_start, t->leaf_start,
                                ((t->adaptive ? t->at.nbox : t->nleaf) + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    return LM_OK;
}

extern "C" lm_status lm_box_export(lm_tree t, int64_t *boxes, int64_t cap, int64_t *count)
{
    if (!t || !count || cap < 0 || (cap > 0 && !boxes)) {
        lm_set_error("box_export: bad argument");
        return LM_EINVAL;
    }
    if (t->adaptive) {
        const int64_t nb = t->at.nbox;
        *count = nb;
        if (cap > 0) memcpy(boxes, t->at.hbox.data(), std::min(cap, nb) * 4 * sizeof(int64_t));
        return LM_OK;
    }
    int64_t e = 0;
    for (int l = 0; l <= t->L; ++l) {
        const int64_t ncol = (int64_t)t->R << l, nrow = (int64_t)1 << l;
        for (int64_t b = 0; b < ncol * nrow; ++b, ++e)
            if (e < cap) {
                boxes[4 * e] = l;
                boxes[4 * e + 1] = b % ncol;
                boxes[4 * e + 2] = b / ncol;
                boxes[4 * e + 3] = l == t->L;
            }
    }
    *count = e;
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
    lm_status s = t->adaptive ? lm_adaptive_lists_to_host(t, which, rows, (cudaStream_t)stream)
                              : lm_list_to_host(t, which, level, rows, (cudaStream_t)stream);
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
    if (t->adaptive) {
        lm_set_error("m2l_table_export: classes of an adaptive tree are not keyed by (level, dc, dr)");
        return LM_ENOTSUP;
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

// ---------------------------------------------------------------------------
// phase profiling: each phase of one apply may be entered several times (per
// level); its events bracket the first begin and the last end of that apply.
// ---------------------------------------------------------------------------
static thread_local int tl_apply_slot = -1;
#define LM_PROF_OCC 24 // event pairs per phase per apply (one per level at most)

// each begin/end pair of a phase gets its own events; the phase total is the
// sum of its pairs, so phases that interleave level by level are not double counted
void lm_phase_begin(lm_tree_s *t, int ph, cudaStream_t st)
{
    if (t->prof_max == 0 || tl_apply_slot < 0) return;
    int occ = t->prof_occ[ph];
    if (occ >= LM_PROF_OCC) return;
    cudaEventRecord(t->prof_ev[(((size_t)tl_apply_slot * LM_NPHASE + ph) * LM_PROF_OCC + occ) * 2], st);
}
void lm_phase_end(lm_tree_s *t, int ph, cudaStream_t st, int launches)
{
    if (t->prof_max == 0 || tl_apply_slot < 0) return;
    int occ = t->prof_occ[ph];
    if (occ >= LM_PROF_OCC) return;
    cudaEventRecord(t->prof_ev[(((size_t)tl_apply_slot * LM_NPHASE + ph) * LM_PROF_OCC + occ) * 2 + 1], st);
    t->prof_occ[ph] = occ + 1;
    t->prof_launch[ph] += launches;
}

void lm_profile_apply_start(lm_tree_s *t)
{
    tl_apply_slot = -1;
    if (t->prof_max > 0 && t->prof_used < t->prof_max) {
        tl_apply_slot = t->prof_used++;
        for (int i = 0; i < 8; ++i) t->prof_occ[i] = 0;
    }
}
void lm_profile_apply_stop(lm_tree_s *t)
{
    if (tl_apply_slot >= 0)
        for (int i = 0; i < LM_NPHASE; ++i) t->prof_nocc[(size_t)tl_apply_slot * LM_NPHASE + i] = t->prof_occ[i];
    tl_apply_slot = -1;
}

extern "C" lm_status lm_profile_begin(lm_tree t, int max_applies)
{
    if (!t || max_applies < 1) {
        lm_set_error("profile_begin: bad argument");
        return LM_EINVAL;
    }
    for (cudaEvent_t e : t->prof_ev) cudaEventDestroy(e);
    t->prof_ev.assign((size_t)max_applies * LM_NPHASE * LM_PROF_OCC * 2, nullptr);
    for (auto &e : t->prof_ev) LM_CUDA(cudaEventCreate(&e));
    t->prof_nocc.assign((size_t)max_applies * LM_NPHASE, 0);
    t->prof_max = max_applies;
    t->prof_used = 0;
    for (int i = 0; i < 8; ++i) t->prof_launch[i] = 0;
    return LM_OK;
}

extern "C" lm_status lm_profile_end(lm_tree t, double *ms, int64_t *launches, int nphase, int *applies)
{
    if (!t || t->prof_max == 0) {
        lm_set_error("profile_end: profiling is not enabled");
        return LM_EINVAL;
    }
    std::vector<double> acc(LM_NPHASE, 0.0);
    for (int a = 0; a < t->prof_used; ++a)
        for (int ph = 0; ph < LM_NPHASE; ++ph)
            for (int o = 0; o < t->prof_nocc[(size_t)a * LM_NPHASE + ph]; ++o) {
                cudaEvent_t *ev = &t->prof_ev[(((size_t)a * LM_NPHASE + ph) * LM_PROF_OCC + o) * 2];
                LM_CUDA(cudaEventSynchronize(ev[1]));
                float f = 0.f;
                LM_CUDA(cudaEventElapsedTime(&f, ev[0], ev[1]));
                acc[ph] += f;
            }
    for (int ph = 0; ph < nphase && ph < LM_NPHASE; ++ph) {
        if (ms) ms[ph] = acc[ph];
        if (launches) launches[ph] = t->prof_launch[ph];
    }
    if (applies) *applies = t->prof_used;
    for (cudaEvent_t e : t->prof_ev) cudaEventDestroy(e);
    t->prof_ev.clear();
    t->prof_max = 0;
    t->prof_used = 0;
    return LM_OK;
}

// ---------------------------------------------------------------------------
// peak probe: independent FMA / transcendental chains on every SM
// ---------------------------------------------------------------------------
__global__ void k_probe_f64(int64_t iters, double *sink)
{
    double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, b = 0.999999, c = 1e-7;
    for (int64_t i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c);
        a1 = fma(a1, b, c);
        a2 = fma(a2, b, c);
        a3 = fma(a3, b, c);
    }
    if (a0 + a1 + a2 + a3 == 12345.0) sink[0] = a0;
}
__global__ void k_probe_f32(int64_t iters, float *sink)
{
    float a[8];
    for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 1e-3f + j;
    const float b = 0.999999f, c = 1e-7f;
    for (int64_t i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
    float s = 0.f;
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.f) sink[0] = s;
}
__global__ void k_probe_sfu(int64_t iters, float *sink)
{
    float a0 = threadIdx.x * 1e-3f, a1 = a0 + 0.5f;
    for (int64_t i = 0; i < iters; ++i) {
        a0 = __sinf(a0) + 0.5f;
        a1 = __cosf(a1) + 0.25f;
    }
    if (a0 + a1 == 12345.f) sink[0] = a0;
}
__global__ void k_probe_exp64(int64_t iters, double *sink)
{
    double a0 = threadIdx.x * 1e-6, a1 = a0 + 0.1;
    for (int64_t i = 0; i < iters; ++i) {
        a0 = exp(-a0) * 0.5;
        a1 = exp(-a1) * 0.5;
    }
    if (a0 + a1 == 12345.0) sink[0] = a0;
}

extern "C" lm_status lm_peak_probe(int kind, int64_t iters, void *stream, double *rate)
{
    if (!rate || iters < 1 || kind < 0 || kind > 3) {
        lm_set_error("peak_probe: bad argument");
        return LM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    LM_CUDA(cudaGetDevice(&dev));
    LM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    double *sink;
    LM_CUDA(cudaMalloc(&sink, 64));
    const int threads = 512, blocks = nsm * 4;
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0));
    LM_CUDA(cudaEventCreate(&e1));
    double ops = 0.0;
    for (int rep = 0; rep < 2; ++rep) { // first run warms up
        LM_CUDA(cudaEventRecord(e0, st));
        switch (kind) {
        case 0: k_probe_f64<<<blocks, threads, 0, st>>>(iters, sink); ops = 4.0 * 2; break;
        case 1: k_probe_f32<<<blocks, threads, 0, st>>>(iters, (float *)sink); ops = 8.0 * 2; break;
        case 2: k_probe_sfu<<<blocks, threads, 0, st>>>(iters, (float *)sink); ops = 2.0; break;
        default: k_probe_exp64<<<blocks, threads, 0, st>>>(iters, sink); ops = 2.0; break;
        }
        LM_CUDA(cudaEventRecord(e1, st));
    }
    LM_CUDA(cudaEventSynchronize(e1));
    float msf = 0.f;
    LM_CUDA(cudaEventElapsedTime(&msf, e0, e1));
    *rate = ops * (double)iters * blocks * threads / (msf * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return LM_OK;
}

// ---------------------------------------------------------------------------
// batched apply as one captured CUDA graph
// ---------------------------------------------------------------------------
struct lm_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    lm_tt_batch_s *tiles = nullptr; // one tile-form M2L over every tree (nullptr: per-tree applies)
    int64_t kernels = 0;            // kernel nodes of the captured graph
};

extern "C" void lm_batch_destroy(lm_batch b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    lm_tt_batch_free(b->tiles);
    delete b;
}

extern "C" lm_status lm_batch_create(const lm_tree *trees, int count, const void *const *q, const int *nvec,
                                     void *const *u, const int *c64, lm_batch *out)
{
    if (!out || !trees || !q || !nvec || !u || count < 1) {
        lm_set_error("batch_create: bad argument");
        return LM_EINVAL;
    }
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        const bool f = c64 && c64[i];
        lm_status s = check_apply(trees[i], q[i], nvec[i], u[i], f ? sizeof(zf) : sizeof(zd));
        if (s != LM_OK) return s;
        if (f && trees[i]->precision != LM_MIXED) {
            lm_set_error("batch_create: complex64 buffers of entry %d need an LM_MIXED tree", i);
            return LM_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (trees[j] == trees[i]) { // one tree's scratch cannot serve two concurrent applies
                lm_set_error("batch_create: tree %d appears twice", i);
                return LM_EINVAL;
            }
        if (trees[i]->prof_max) {
            lm_set_error("batch_create: profiling is enabled on tree %d", i);
            return LM_EINVAL;
        }
    }
    const int nstream = std::min(count, 8);
    cudaStream_t cs, side[8];
    cudaEvent_t fork, join[8];
    LM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    for (int k = 0; k < nstream; ++k) {
        LM_CUDA(cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking));
        LM_CUDA(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
    }
    LM_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    lm_batch_s *b = new (std::nothrow) lm_batch_s();
    if (!b) {
        lm_set_error("batch_create: host allocation failed");
        return LM_ENOMEM;
    }
    // One M2L launch for the whole batch when every tree runs the tile form with the
    // same p and vector slots: the trees' upward passes (permute, S2M, M2M, multipole
    // split) run on the side streams, then one persistent tile launch walks the
    // concatenated work list of every tree's tiles, then the downward passes (L2L,
    // leaf step, permute) run on the side streams again.
    bool joint = count >= 2;
    const int nvs0 = nvec[0] <= 4 ? 4 : LM_MAXV;
    for (int i = 0; i < count && joint; ++i)
        joint = lm_mixed_tiles(trees[i], nvec[i]) && trees[i]->p == trees[0]->p &&
                (nvec[i] <= 4 ? 4 : LM_MAXV) == nvs0;
    lm_status st = LM_OK;
    if (joint) {
        std::vector<lm_tree_s *> tv(trees, trees + count);
        st = lm_tt_batch_build(tv.data(), count, nvs0, &b->tiles);
        if (st != LM_OK) {
            lm_batch_destroy(b);
            return st;
        }
    }
    auto capture_part = [&](int part) {
        cudaEventRecord(fork, cs);
        for (int k = 0; k < nstream; ++k) cudaStreamWaitEvent(side[k], fork, 0);
        for (int i = 0; i < count && st == LM_OK; ++i) {
            const bool f = c64 && c64[i];
            st = (f || part != 0)
                     ? lm_run_apply_mixed(trees[i], q[i], nvec[i], u[i], false, f, side[i % nstream], part)
                     : lm_run_apply(trees[i], (const zd *)q[i], nvec[i], (zd *)u[i], false, side[i % nstream]);
            if (st != LM_OK) {
                std::string why = lm_last_error();
                lm_set_error("batch_create: capturing the apply of tree %d failed: %s", i, why.c_str());
            }
        }
        for (int k = 0; k < nstream; ++k) {
            cudaEventRecord(join[k], side[k]);
            cudaStreamWaitEvent(cs, join[k], 0);
        }
    };
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (joint) {
            capture_part(1);
            if (st == LM_OK) st = lm_tt_batch_launch(b->tiles, cs);
            if (st == LM_OK) capture_part(2);
        } else {
            capture_part(0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
        if (st == LM_OK && e2 != cudaSuccess) {
            lm_set_error("batch_create: capture failed: %s", cudaGetErrorString(e2));
            st = LM_ECUDA;
        }
        if (st == LM_OK) {
            size_t nn = 0;
            e2 = cudaGraphGetNodes(b->graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (e2 == cudaSuccess && nn) e2 = cudaGraphGetNodes(b->graph, nodes.data(), &nn);
            for (size_t i = 0; i < nn && e2 == cudaSuccess; ++i) {
                cudaGraphNodeType ty;
                e2 = cudaGraphNodeGetType(nodes[i], &ty);
                b->kernels += ty == cudaGraphNodeTypeKernel;
            }
            if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e2 != cudaSuccess) {
                lm_set_error("batch_create: graph instantiation failed: %s", cudaGetErrorString(e2));
                st = LM_ECUDA;
            }
        }
    } else {
        lm_set_error("batch_create: cudaStreamBeginCapture failed: %s", cudaGetErrorString(e));
        st = LM_ECUDA;
    }
    cudaEventDestroy(fork);
    for (int k = 0; k < nstream; ++k) {
        cudaEventDestroy(join[k]);
        cudaStreamDestroy(side[k]);
    }
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (st != LM_OK) {
        lm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LM_OK;
}

extern "C" lm_status lm_batch_launch(lm_batch b, void *stream)
{
    if (!b || !b->exec) {
        lm_set_error("batch_launch: NULL batch");
        return LM_EINVAL;
    }
    LM_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return LM_OK;
}

extern "C" lm_status lm_batch_info(lm_batch b, int64_t *kernels, int *joint_m2l)
{
    if (!b) {
        lm_set_error("batch_info: NULL batch");
        return LM_EINVAL;
    }
    if (kernels) *kernels = b->kernels;
    if (joint_m2l) *joint_m2l = b->tiles != nullptr;
    return LM_OK;
}

// ---------------------------------------------------------------------------
// monotone dynamic shared-memory limits (per device, per kernel slot)
// ---------------------------------------------------------------------------
#define LM_SMEM_MAXDEV 64
static int g_smem_set[LM_SMEM_MAXDEV][LM_SMEM_SLOTS];
static std::mutex g_smem_mutex;

cudaError_t lm_raise_smem(const void *func, int slot, int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= LM_SMEM_MAXDEV || slot < 0 || slot >= LM_SMEM_SLOTS)
        return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    if (bytes <= g_smem_set[dev][slot]) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) g_smem_set[dev][slot] = bytes;
    return e;
}
