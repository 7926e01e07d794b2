// lmfmm_noalloc.cu -- lm_tree_order_noalloc: the tree order of lm_build_tree
// computed without allocating memory, for callers that cannot allocate.
//
// Its scratch lives in one file-scope device array of fixed size below; every
// GPU that loads the library holds it until the process exits.  Host code
// never dereferences or passes the array's name: on first use on a device
// (with that device current) the entry point asks the runtime for the
// array's device address and caches it per device.  A device reset reloads
// the module and may move the array, so the cache is not valid across one.
#include <cmath>
#include <mutex>

#include "internal.h"

// limits of the allocation-free path
#define NA_MAXN (1 << 20)    // points
#define NA_MAXLEAF (1 << 18) // leaves (R 4^L)
#define NA_MAXBLK 1024       // blocks of the extent reduction
#define NA_MAXDEV 64

// scratch layout: keys [NA_MAXN] int32 | counts [NA_MAXLEAF] int32 |
// cursors [NA_MAXLEAF] int32 | block minima [NA_MAXBLK] double | block maxima
// [NA_MAXBLK] double | flags [4] int
#define NA_OFF_KEY 0
#define NA_OFF_CNT (NA_OFF_KEY + (size_t)NA_MAXN * 4)
#define NA_OFF_CUR (NA_OFF_CNT + (size_t)NA_MAXLEAF * 4)
#define NA_OFF_MIN (NA_OFF_CUR + (size_t)NA_MAXLEAF * 4)
#define NA_OFF_MAX (NA_OFF_MIN + (size_t)NA_MAXBLK * 8)
#define NA_OFF_FLAG (NA_OFF_MAX + (size_t)NA_MAXBLK * 8)
#define NA_BYTES (NA_OFF_FLAG + 16)

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

static unsigned char *g_na_ptr[NA_MAXDEV];
static std::mutex g_na_mutex;

// kernels shared with lm_build_tree (lmfmm_setup.cu)
__global__ void k_minmax(const double *x, const double *y, int64_t n, double d, double *bmin, double *bmax,
                         int *flag);
__global__ void k_keys(const double *x, const double *y, int64_t n, double x0, double w, int64_t ncol,
                       int64_t nrow, int32_t *key, int32_t *cnt);
__global__ void k_scan(const int32_t *cnt, int64_t m, int64_t *start);
__global__ void k_scatter(const int32_t *key, int64_t n, const int64_t *start, int32_t *cursor, int64_t *tmp);
__global__ void k_leafsort(const int64_t *start, int64_t *idx, int *flag);

// device address of the scratch array on the current device (set-up on first use)
static lm_status na_scratch(unsigned char **out)
{
    int dev = 0;
    LM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAXDEV) {
        lm_set_error("tree_order_noalloc: device %d beyond %d", dev, NA_MAXDEV);
        return LM_ENOTSUP;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            lm_set_error("tree_order_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return LM_ECUDA;
        }
        g_na_ptr[dev] = (unsigned char *)p;
    }
    *out = g_na_ptr[dev];
    return LM_OK;
}

extern "C" lm_status lm_tree_order_noalloc(const double *x, const double *y, int64_t n, double d, int depth,
                                           int64_t *perm, int64_t *leaf_start, int64_t leaf_cap,
                                           double *x_origin, int *R, void *stream)
{
    if (!x || !y || !perm || !leaf_start || !x_origin || !R) {
        lm_set_error("tree_order_noalloc: NULL pointer argument");
        return LM_EINVAL;
    }
    if (n < 1 || n > NA_MAXN) {
        lm_set_error("tree_order_noalloc: n = %lld outside 1..%d (the fixed scratch limit)", (long long)n,
                     NA_MAXN);
        return LM_EINVAL;
    }
    if (!(d > 0.0) || !std::isfinite(d) || depth < 0 || depth > 14) {
        lm_set_error("tree_order_noalloc: need a finite d > 0 and depth in 0..14");
        return LM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *s = nullptr;
    lm_status ss = na_scratch(&s);
    if (ss != LM_OK) return ss;
    int32_t *key = (int32_t *)(s + NA_OFF_KEY), *cnt = (int32_t *)(s + NA_OFF_CNT),
            *cur = (int32_t *)(s + NA_OFF_CUR);
    double *bmin = (double *)(s + NA_OFF_MIN), *bmax = (double *)(s + NA_OFF_MAX);
    int *flag = (int *)(s + NA_OFF_FLAG);

    // extent along x and point validity (same reduction as lm_build_tree)
    const int nb = (int)std::min<int64_t>(NA_MAXBLK, (n + 255) / 256);
    LM_CUDA(cudaMemsetAsync(flag, 0, 4 * sizeof(int), st));
    k_minmax<<<nb, 256, 0, st>>>(x, y, n, d, bmin, bmax, flag);
    double hmin[NA_MAXBLK], hmax[NA_MAXBLK];
    int hflag = 0;
    LM_CUDA(cudaMemcpyAsync(hmin, bmin, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(hmax, bmax, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    if (hflag & 1) {
        lm_set_error("tree_order_noalloc: a point is non-finite or not strictly inside -d < y < 0");
        return LM_EINVAL;
    }
    double mn = hmin[0], mx = hmax[0];
    for (int i = 1; i < nb; ++i) {
        mn = fmin(mn, hmin[i]);
        mx = fmax(mx, hmax[i]);
    }
    const double f0 = floor(mn / d), f1 = floor(mx / d);
    // leaves counted in double before any integer conversion, so that a huge x
    // extent (or a tiny d) cannot wrap the root count
    const double dleaf = (f1 - f0 + 1.0) * ldexp(1.0, 2 * depth);
    if (!std::isfinite(dleaf) || dleaf > (double)NA_MAXLEAF) {
        lm_set_error("tree_order_noalloc: %g leaves exceed the fixed scratch limit of %d", dleaf, NA_MAXLEAF);
        return LM_EINVAL;
    }
    const int Rv = (int)(f1 - f0) + 1;
    const int64_t ncol = (int64_t)Rv << depth, nrow = (int64_t)1 << depth, nleaf = ncol * nrow;
    if (leaf_cap < nleaf + 1) {
        lm_set_error("tree_order_noalloc: leaf_start holds %lld entries, %lld needed", (long long)leaf_cap,
                     (long long)(nleaf + 1));
        *R = Rv;
        *x_origin = f0 * d;
        return LM_EINVAL;
    }
    // the array keeps the previous call's contents: clear what must start at zero
    LM_CUDA(cudaMemsetAsync(cnt, 0, nleaf * sizeof(int32_t), st));
    LM_CUDA(cudaMemsetAsync(cur, 0, nleaf * sizeof(int32_t), st));
    const double x0 = f0 * d, w = ldexp(d, -depth);
    const int g = (int)((n + 255) / 256);
    k_keys<<<g, 256, 0, st>>>(x, y, n, x0, w, ncol, nrow, key, cnt);
    k_scan<<<1, 1024, 0, st>>>(cnt, nleaf, leaf_start);
    k_scatter<<<g, 256, 0, st>>>(key, n, leaf_start, cur, perm);
    k_leafsort<<<(unsigned)nleaf, 256, 0, st>>>(leaf_start, perm, flag);
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    if (hflag & 2) {
        lm_set_error("tree_order_noalloc: a leaf holds more than %d points; use a deeper tree", LM_MAXLEAF);
        return LM_ENOTSUP;
    }
    *x_origin = x0;
    *R = Rv;
    return LM_OK;
}
