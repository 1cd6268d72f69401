// tables.cu -- the library-owned lookup tables (§3.1, §3.2): creation from host
// arrays, FP32 copies (§3.3: computed in double, stored in single), views for
// kernels, host copies, and a checked binary file format.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "physics.cuh"

namespace qed {

static qed_status check_axis(const qed_table_axis &a, const char *name, bool qs)
{
    if (!(a.chi_min > 0.0) || !(a.chi_max > a.chi_min) || !std::isfinite(a.chi_max))
        QED_FAIL(QED_ERR_INVALID_ARG, "%s: need 0 < chi_min < chi_max (got %g, %g)", name, a.chi_min, a.chi_max);
    if (a.n_chi < 2 || a.n_chi > QED_MAX_TABLE_N || a.n_xi < 2 || a.n_xi > QED_MAX_TABLE_N)
        QED_FAIL(QED_ERR_INVALID_ARG, "%s: n_chi, n_xi must be in [2, %d] (got %d, %d)", name, QED_MAX_TABLE_N, a.n_chi, a.n_xi);
    if (qs && !(a.xi_min > 0.0 && a.xi_min < 1.0))
        QED_FAIL(QED_ERR_INVALID_ARG, "%s: need 0 < xi_min < 1 (got %g)", name, a.xi_min);
    return QED_OK;
}

qed_status check_params(const qed_table_params *p)
{
    if (p == nullptr) QED_FAIL(QED_ERR_INVALID_ARG, "params is NULL");
    qed_status s = check_axis(p->qs, "qs", true);
    if (s) return s;
    return check_axis(p->bw, "bw", false);
}

// d[n][m] = v[n][m+1] - v[n][m] in FP64, 0 in the last column
__global__ void col_diff_kernel(const double *__restrict__ v, double *__restrict__ d, int64_t rows, int cols)
{
    const int64_t n = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % cols);
        d[i] = (m + 1 < cols) ? v[i + 1] - v[i] : 0.0;
    }
}

__global__ void to_f32_kernel(const double *__restrict__ in, float *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

// Guide table of one 2-D table: for row n and edge e of kGuideBins equal bins
// of the draw r (QS: r in (0, 1], searched as ln r; BW: r in [0, 1/2]), the
// largest m with v[n][m] <= edge (0 if none); edge 0 is -inf, the last +inf.
// A draw in bin b then lies between the rows' guides at b and b + 1.
template <typename T>
__global__ void guide_kernel(const T *__restrict__ v, int n_xi, bool qs, int32_t *__restrict__ g)
{
    const int n = blockIdx.x, e = threadIdx.x;
    if (e > kGuideBins) return;
    int32_t out;
    if (e == 0) {
        out = 0;
    } else if (e == kGuideBins) {
        out = n_xi - 1;
    } else {
        const T x = qs ? d_log(T(e) / T(kGuideBins)) : T(e) / T(2 * kGuideBins);
        const T *row = v + (size_t)n * n_xi;
        int lo = 0, hi = n_xi;  // largest m with row[m] <= x: row[lo] <= x (or lo == 0), row[hi] > x
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (row[mid] <= x)
                lo = mid;
            else
                hi = mid;
        }
        out = lo;
    }
    g[(size_t)n * (kGuideBins + 1) + e] = out;
}

static void free_tables(qed_tables *t)
{
    if (!t) return;
    void *ptrs[] = {t->d_qs_lnG, t->d_qs_lnP, t->d_bw_lnT, t->d_bw_P, t->f_qs_lnG, t->f_qs_lnP, t->f_bw_lnT, t->f_bw_P,
                    t->d_qs_dlnP, t->d_bw_dP, t->f_qs_dlnP, t->f_bw_dP, t->d_qs_guide, t->d_bw_guide,
                    t->f_qs_guide, t->f_bw_guide};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete t;
}

static size_t n_qs2(const qed_table_params &p) { return (size_t)p.qs.n_chi * p.qs.n_xi; }
static size_t n_bw2(const qed_table_params &p) { return (size_t)p.bw.n_chi * p.bw.n_xi; }

qed_status alloc_tables(const qed_table_params *p, qed_tables **out)
{
    qed_tables *t = new qed_tables();
    memset(t, 0, sizeof(*t));
    t->params = *p;
    cudaGetDevice(&t->device);
    const size_t sz[6] = {(size_t)p->qs.n_chi, n_qs2(*p), (size_t)p->bw.n_chi, n_bw2(*p), n_qs2(*p), n_bw2(*p)};
    double **dp[6] = {&t->d_qs_lnG, &t->d_qs_lnP, &t->d_bw_lnT, &t->d_bw_P, &t->d_qs_dlnP, &t->d_bw_dP};
    float **fp[6] = {&t->f_qs_lnG, &t->f_qs_lnP, &t->f_bw_lnT, &t->f_bw_P, &t->f_qs_dlnP, &t->f_bw_dP};
    for (int k = 0; k < 6; ++k) {
        cudaError_t e1 = cudaMalloc((void **)dp[k], sz[k] * sizeof(double));
        cudaError_t e2 = cudaMalloc((void **)fp[k], sz[k] * sizeof(float));
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            free_tables(t);
            QED_FAIL(QED_ERR_CUDA, "table allocation failed: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        }
    }
    const size_t ng[2] = {(size_t)p->qs.n_chi * (kGuideBins + 1), (size_t)p->bw.n_chi * (kGuideBins + 1)};
    int32_t **gp[4] = {&t->d_qs_guide, &t->f_qs_guide, &t->d_bw_guide, &t->f_bw_guide};
    for (int k = 0; k < 4; ++k) {
        cudaError_t e = cudaMalloc((void **)gp[k], ng[k / 2] * sizeof(int32_t));
        if (e != cudaSuccess) {
            free_tables(t);
            QED_FAIL(QED_ERR_CUDA, "table allocation failed: %s", cudaGetErrorString(e));
        }
    }
    *out = t;
    return QED_OK;
}

// round the FP64 tables into the FP32 copies on `stream`, then the guides
qed_status finish_tables(qed_tables *t, cudaStream_t st)
{
    const qed_table_params &p = t->params;
    col_diff_kernel<<<256, 256, 0, st>>>(t->d_qs_lnP, t->d_qs_dlnP, p.qs.n_chi, p.qs.n_xi);
    QED_LAUNCH_CHECK();
    col_diff_kernel<<<256, 256, 0, st>>>(t->d_bw_P, t->d_bw_dP, p.bw.n_chi, p.bw.n_xi);
    QED_LAUNCH_CHECK();
    const size_t sz[6] = {(size_t)p.qs.n_chi, n_qs2(p), (size_t)p.bw.n_chi, n_bw2(p), n_qs2(p), n_bw2(p)};
    const double *d[6] = {t->d_qs_lnG, t->d_qs_lnP, t->d_bw_lnT, t->d_bw_P, t->d_qs_dlnP, t->d_bw_dP};
    float *f[6] = {t->f_qs_lnG, t->f_qs_lnP, t->f_bw_lnT, t->f_bw_P, t->f_qs_dlnP, t->f_bw_dP};
    for (int k = 0; k < 6; ++k) {
        int blocks = (int)((sz[k] + 255) / 256);
        if (blocks > 1024) blocks = 1024;
        to_f32_kernel<<<blocks, 256, 0, st>>>(d[k], f[k], (int64_t)sz[k]);
        QED_LAUNCH_CHECK();
    }
    guide_kernel<double><<<p.qs.n_chi, kGuideBins + 1, 0, st>>>(t->d_qs_lnP, p.qs.n_xi, true, t->d_qs_guide);
    guide_kernel<float><<<p.qs.n_chi, kGuideBins + 1, 0, st>>>(t->f_qs_lnP, p.qs.n_xi, true, t->f_qs_guide);
    guide_kernel<double><<<p.bw.n_chi, kGuideBins + 1, 0, st>>>(t->d_bw_P, p.bw.n_xi, false, t->d_bw_guide);
    guide_kernel<float><<<p.bw.n_chi, kGuideBins + 1, 0, st>>>(t->f_bw_P, p.bw.n_xi, false, t->f_bw_guide);
    QED_LAUNCH_CHECK();
    QED_CUDA_TRY(cudaStreamSynchronize(st));
    return QED_OK;
}

template <typename T>
static Table1D<T> view1(const T *f, const qed_table_axis &a)
{
    Table1D<T> v;
    v.ln_f = f;
    const double l0 = std::log(a.chi_min), l1 = std::log(a.chi_max);
    v.ln_min = (T)l0;
    v.inv_d = (T)((a.n_chi - 1) / (l1 - l0));
    v.chi_min = (T)a.chi_min;
    v.chi_max = (T)a.chi_max;
    v.n = a.n_chi;
    return v;
}

template <typename T>
static Table2D<T> view2(const T *f, const T *df, const int32_t *guide, const qed_table_axis &a, bool qs)
{
    Table2D<T> v;
    v.v = f;
    v.dv = df;
    v.guide = guide;
    const double l0 = std::log(a.chi_min), l1 = std::log(a.chi_max);
    v.ln_min = (T)l0;
    v.inv_d = (T)((a.n_chi - 1) / (l1 - l0));
    v.chi_min = (T)a.chi_min;
    v.chi_max = (T)a.chi_max;
    v.n_chi = a.n_chi;
    v.n_xi = a.n_xi;
    if (qs) {
        v.x0 = (T)std::log(a.xi_min);
        v.dx = (T)(-std::log(a.xi_min) / (a.n_xi - 1));
    } else {
        v.x0 = (T)0;
        v.dx = (T)(0.5 / (a.n_xi - 1));
    }
    return v;
}

template <>
TablesView<double> make_view<double>(const qed_tables *t)
{
    TablesView<double> v;
    v.qs_G = view1<double>(t->d_qs_lnG, t->params.qs);
    v.bw_T = view1<double>(t->d_bw_lnT, t->params.bw);
    v.qs_P = view2<double>(t->d_qs_lnP, t->d_qs_dlnP, t->d_qs_guide, t->params.qs, true);
    v.bw_P = view2<double>(t->d_bw_P, t->d_bw_dP, t->d_bw_guide, t->params.bw, false);
    return v;
}

template <>
TablesView<float> make_view<float>(const qed_tables *t)
{
    TablesView<float> v;
    v.qs_G = view1<float>(t->f_qs_lnG, t->params.qs);
    v.bw_T = view1<float>(t->f_bw_lnT, t->params.bw);
    v.qs_P = view2<float>(t->f_qs_lnP, t->f_qs_dlnP, t->f_qs_guide, t->params.qs, true);
    v.bw_P = view2<float>(t->f_bw_P, t->f_bw_dP, t->f_bw_guide, t->params.bw, false);
    return v;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_tables_create(const qed_table_params *params, const double *qs_lnG,
                                        const double *qs_lnP, const double *bw_lnT,
                                        const double *bw_P, qed_tables **out, void *stream)
{
    clear_error();
    if (out == nullptr) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    qed_status s = check_params(params);
    if (s) return s;
    if (!qs_lnG || !qs_lnP || !bw_lnT || !bw_P) QED_FAIL(QED_ERR_INVALID_ARG, "a table array is NULL");
    qed_tables *t = nullptr;
    if ((s = alloc_tables(params, &t))) return s;
    cudaStream_t st = as_stream(stream);
    const qed_table_params &p = *params;
    const size_t sz[4] = {(size_t)p.qs.n_chi, n_qs2(p), (size_t)p.bw.n_chi, n_bw2(p)};
    const double *src[4] = {qs_lnG, qs_lnP, bw_lnT, bw_P};
    double *dst[4] = {t->d_qs_lnG, t->d_qs_lnP, t->d_bw_lnT, t->d_bw_P};
    for (int k = 0; k < 4; ++k) {
        cudaError_t e = cudaMemcpyAsync(dst[k], src[k], sz[k] * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            free_tables(t);
            QED_FAIL(QED_ERR_CUDA, "table upload failed: %s", cudaGetErrorString(e));
        }
    }
    if ((s = finish_tables(t, st))) {
        free_tables(t);
        return s;
    }
    *out = t;
    return QED_OK;
}

extern "C" qed_status qed_tables_copy_to_host(const qed_tables *t, double *qs_lnG, double *qs_lnP,
                                              double *bw_lnT, double *bw_P)
{
    clear_error();
    qed_status s = check_tables(t);
    if (s) return s;
    const qed_table_params &p = t->params;
    const size_t sz[4] = {(size_t)p.qs.n_chi, n_qs2(p), (size_t)p.bw.n_chi, n_bw2(p)};
    const double *src[4] = {t->d_qs_lnG, t->d_qs_lnP, t->d_bw_lnT, t->d_bw_P};
    double *dst[4] = {qs_lnG, qs_lnP, bw_lnT, bw_P};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) QED_CUDA_TRY(cudaMemcpy(dst[k], src[k], sz[k] * sizeof(double), cudaMemcpyDeviceToHost));
    return QED_OK;
}

extern "C" qed_status qed_tables_get_params(const qed_tables *t, qed_table_params *out)
{
    clear_error();
    qed_status s = check_tables(t);
    if (s) return s;
    if (!out) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    *out = t->params;
    return QED_OK;
}

extern "C" qed_status qed_tables_destroy(qed_tables *t)
{
    clear_error();
    free_tables(t);
    return QED_OK;
}

// ---------------------------------------------------------------------------
// file format: "QEDTAB\0\1" | u32 version | params (5 doubles/ints per axis) |
// qs_lnG | qs_lnP | bw_lnT | bw_P (FP64, little-endian host order) | u64 FNV-1a
// ---------------------------------------------------------------------------
static const char kMagic[8] = {'Q', 'E', 'D', 'T', 'A', 'B', 0, 1};
static const uint32_t kFileVersion = 1;

static void put_axis(std::vector<unsigned char> &buf, const qed_table_axis &a)
{
    auto put = [&](const void *p, size_t n) { buf.insert(buf.end(), (const unsigned char *)p, (const unsigned char *)p + n); };
    put(&a.chi_min, 8);
    put(&a.chi_max, 8);
    put(&a.n_chi, 4);
    put(&a.n_xi, 4);
    put(&a.xi_min, 8);
}

extern "C" qed_status qed_tables_save(const qed_tables *t, const char *path)
{
    clear_error();
    qed_status s = check_tables(t);
    if (s) return s;
    if (!path) QED_FAIL(QED_ERR_INVALID_ARG, "path is NULL");
    const qed_table_params &p = t->params;
    std::vector<double> a(p.qs.n_chi), b(n_qs2(p)), c(p.bw.n_chi), d(n_bw2(p));
    if ((s = qed_tables_copy_to_host(t, a.data(), b.data(), c.data(), d.data()))) return s;
    std::vector<unsigned char> buf;
    buf.insert(buf.end(), kMagic, kMagic + 8);
    buf.insert(buf.end(), (const unsigned char *)&kFileVersion, (const unsigned char *)&kFileVersion + 4);
    put_axis(buf, p.qs);
    put_axis(buf, p.bw);
    for (auto *v : {&a, &b, &c, &d})
        buf.insert(buf.end(), (const unsigned char *)v->data(), (const unsigned char *)(v->data() + v->size()));
    const uint64_t h = fnv1a64(buf.data(), buf.size());
    FILE *f = fopen(path, "wb");
    if (!f) QED_FAIL(QED_ERR_IO, "cannot open %s for writing", path);
    bool ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size() && fwrite(&h, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok) QED_FAIL(QED_ERR_IO, "write to %s failed", path);
    return QED_OK;
}

extern "C" qed_status qed_tables_load(const char *path, qed_tables **out, void *stream)
{
    clear_error();
    if (!path || !out) QED_FAIL(QED_ERR_INVALID_ARG, "path/out is NULL");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) QED_FAIL(QED_ERR_IO, "cannot open %s", path);
    std::vector<unsigned char> buf;
    unsigned char chunk[1 << 16];
    size_t n;
    while ((n = fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + n);
    fclose(f);
    const size_t head = 8 + 4 + 2 * 32;
    if (buf.size() < head + 8) QED_FAIL(QED_ERR_IO, "%s: file too short", path);
    if (memcmp(buf.data(), kMagic, 8) != 0) QED_FAIL(QED_ERR_IO, "%s: bad magic", path);
    uint32_t ver;
    memcpy(&ver, buf.data() + 8, 4);
    if (ver != kFileVersion) QED_FAIL(QED_ERR_IO, "%s: unsupported version %u", path, ver);
    qed_table_params p;
    const unsigned char *q = buf.data() + 12;
    for (qed_table_axis *a : {&p.qs, &p.bw}) {
        memcpy(&a->chi_min, q, 8);
        memcpy(&a->chi_max, q + 8, 8);
        memcpy(&a->n_chi, q + 16, 4);
        memcpy(&a->n_xi, q + 20, 4);
        memcpy(&a->xi_min, q + 24, 8);
        q += 32;
    }
    qed_status s = check_params(&p);
    if (s) QED_FAIL(QED_ERR_IO, "%s: bad table parameters", path);
    const size_t body = 8 * ((size_t)p.qs.n_chi + n_qs2(p) + (size_t)p.bw.n_chi + n_bw2(p));
    if (buf.size() != head + body + 8) QED_FAIL(QED_ERR_IO, "%s: size mismatch", path);
    uint64_t h;
    memcpy(&h, buf.data() + head + body, 8);
    if (h != fnv1a64(buf.data(), head + body)) QED_FAIL(QED_ERR_IO, "%s: checksum mismatch", path);
    const double *d = (const double *)(buf.data() + head);
    std::vector<double> arr(body / 8);
    memcpy(arr.data(), d, body);
    const double *a0 = arr.data();
    const double *a1 = a0 + p.qs.n_chi;
    const double *a2 = a1 + n_qs2(p);
    const double *a3 = a2 + p.bw.n_chi;
    return qed_tables_create(&p, a0, a1, a2, a3, out, stream);
}
