// lmfmm_grad.cu -- lm_misfit_grad: every gradient of a real misfit J(u),
// u = G(x, y, d) q, assembled on the device from the FMM applies.
//
// With g = dJ/d(Re u) + i dJ/d(Im u) (the adjoint input a caller's autodiff
// hands back):
//   dJ/dq   = G^H g = conj(G conj g)                     (reciprocity, Sec. 3)
//   dJ/dx_j = Re sum_v [conj(g_vj) dx(G q_v)_j + q_vj dx(G conj g_v)_j]
//   dJ/dy_j = the same with dy
//   dJ/dd   = Re sum_v sum_i conj(g_vi) (dG/dd q_v)_i
// The two x (y) terms are the target gradient of G at x_j applied to q and the
// target gradient applied to conj g, which by G(a, b) = G(b, a) is the
// derivative in the source point; both come from one lm_apply_grad over the
// stacked vectors [q; conj g].  dG/dd comes from a tree built with
// kernel = LM_KERNEL_DG_DD over the same points.  The d-sum is reduced in a
// fixed order (per-block partials, then one block), so it is reproducible.
#include "internal.h"

static int gridg(int64_t n, int b) { return (int)((n + b - 1) / b); }

// V = [q; conj g], [2 nvec][n]
__global__ void k_stack_conj(const zd *q, const zd *g, int64_t n, int nvec, zd *V)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)nvec * n) return;
    V[i] = q[i];
    V[(int64_t)nvec * n + i] = conj(g[i]);
}

// gx_j = Re sum_v [conj(g_vj) UX[v][j] + q_vj UX[nvec + v][j]], gy likewise
__global__ void k_grad_xy(const zd *q, const zd *g, const zd *UX, const zd *UY, int64_t n, int nvec, double *gx,
                          double *gy)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sx = 0.0, sy = 0.0;
    for (int v = 0; v < nvec; ++v) {
        const int64_t a = (int64_t)v * n + j, b = (int64_t)(nvec + v) * n + j;
        const zd gc = conj(g[a]), qv = q[a];
        if (gx) sx += (gc * UX[a] + qv * UX[b]).re;
        if (gy) sy += (gc * UY[a] + qv * UY[b]).re;
    }
    if (gx) gx[j] = sx;
    if (gy) gy[j] = sy;
}

#define GD_THREADS 256
#define GD_BLOCKS 256
// partial[b] = Re sum over the block's share of conj(g) * DD, in a fixed order
__global__ void __launch_bounds__(GD_THREADS) k_grad_d_partial(const zd *g, const zd *DD, int64_t m, double *partial)
{
    __shared__ double s[GD_THREADS];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)GD_THREADS + threadIdx.x; i < m; i += (int64_t)GD_BLOCKS * GD_THREADS)
        acc += (conj(g[i]) * DD[i]).re;
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = GD_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}
__global__ void __launch_bounds__(GD_THREADS) k_grad_d_final(const double *partial, double *gd)
{
    __shared__ double s[GD_THREADS];
    s[threadIdx.x] = threadIdx.x < GD_BLOCKS ? partial[threadIdx.x] : 0.0;
    __syncthreads();
    for (int w = GD_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *gd = s[0];
}

// workspace: V [2 nvec][n] | UX [2 nvec][n] | UY [2 nvec][n] | DD [nvec][n] | partials [GD_BLOCKS]
static size_t grad_ws_bytes(int64_t n, int nvec)
{
    return ((size_t)7 * nvec * n) * sizeof(zd) + GD_BLOCKS * sizeof(double);
}

extern "C" lm_status lm_misfit_grad_workspace(lm_tree t, int nvec, size_t *bytes)
{
    if (!t || nvec < 1 || !bytes) {
        lm_set_error("misfit_grad_workspace: NULL tree or output, or nvec < 1");
        return LM_EINVAL;
    }
    *bytes = grad_ws_bytes(t->n, nvec);
    return LM_OK;
}

static bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    if (!a || !b) return false;
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

extern "C" lm_status lm_misfit_grad(lm_tree t, lm_tree dtree, const void *q, const void *g, int nvec, void *gq,
                                    double *gx, double *gy, double *gd, void *workspace, size_t ws_bytes,
                                    void *stream)
{
    if (!t || !q || !g || nvec < 1) {
        lm_set_error("misfit_grad: NULL tree, q or g, or nvec < 1");
        return LM_EINVAL;
    }
    const int64_t n = t->n;
    const size_t vb = (size_t)nvec * n * sizeof(zd);
    const bool xy = gx || gy;
    if ((xy || gd) && (!workspace || ws_bytes < grad_ws_bytes(n, nvec))) {
        lm_set_error("misfit_grad: workspace of %zu bytes, %zu needed", ws_bytes, grad_ws_bytes(n, nvec));
        return LM_EINVAL;
    }
    if (xy && t->precision != LM_FP64) {
        lm_set_error("misfit_grad: coordinate gradients need an LM_FP64 tree");
        return LM_ENOTSUP;
    }
    if (gd && (!dtree || dtree->n != n || dtree->med.opt.kernel != LM_KERNEL_DG_DD)) {
        lm_set_error("misfit_grad: d-gradient needs the dG/dd tree of the same points");
        return LM_EINVAL;
    }
    const size_t ws = grad_ws_bytes(n, nvec);
    const void *outs[] = {gq, gx, gy, gd};
    const size_t outb[] = {vb, n * sizeof(double), n * sizeof(double), sizeof(double)};
    for (int a = 0; a < 4; ++a) {
        if (overlaps(outs[a], outb[a], q, vb) || overlaps(outs[a], outb[a], g, vb) ||
            overlaps(outs[a], outb[a], workspace, ws)) {
            lm_set_error("misfit_grad: an output overlaps an input or the workspace");
            return LM_EINVAL;
        }
        for (int b = 0; b < a; ++b)
            if (overlaps(outs[a], outb[a], outs[b], outb[b])) {
                lm_set_error("misfit_grad: outputs overlap");
                return LM_EINVAL;
            }
    }
    cudaStream_t st = (cudaStream_t)stream;
    zd *V = (zd *)workspace, *UX = V + (size_t)2 * nvec * n, *UY = UX + (size_t)2 * nvec * n;
    zd *DD = UY + (size_t)2 * nvec * n;
    double *partial = (double *)(DD + (size_t)nvec * n);
    lm_status s = LM_OK;
    if (gq) {
        lm_profile_apply_start(t);
        s = lm_run_apply(t, (const zd *)g, nvec, (zd *)gq, true, st);
        lm_profile_apply_stop(t);
        if (s != LM_OK) return s;
    }
    if (xy) {
        k_stack_conj<<<gridg((int64_t)nvec * n, 256), 256, 0, st>>>((const zd *)q, (const zd *)g, n, nvec, V);
        lm_profile_apply_start(t);
        s = lm_run_apply_grad(t, V, 2 * nvec, nullptr, UX, UY, st);
        lm_profile_apply_stop(t);
        if (s != LM_OK) return s;
        k_grad_xy<<<gridg(n, 256), 256, 0, st>>>((const zd *)q, (const zd *)g, UX, UY, n, nvec, gx, gy);
    }
    if (gd) {
        lm_profile_apply_start(dtree);
        s = lm_run_apply(dtree, (const zd *)q, nvec, DD, false, st);
        lm_profile_apply_stop(dtree);
        if (s != LM_OK) return s;
        k_grad_d_partial<<<GD_BLOCKS, GD_THREADS, 0, st>>>((const zd *)g, DD, (int64_t)nvec * n, partial);
        k_grad_d_final<<<1, GD_THREADS, 0, st>>>(partial, gd);
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}
