// capi.cu -- error reporting, version and argument validation of the C ABI.
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace qed {

static thread_local char g_err[1024] = {0};

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

qed_status check_tables(const qed_tables *t)
{
    if (t == nullptr) QED_FAIL(QED_ERR_INVALID_ARG, "tables handle is NULL");
    if (!t->d_qs_lnG || !t->f_qs_lnG) QED_FAIL(QED_ERR_INVALID_ARG, "tables handle is not initialised");
    return QED_OK;
}

qed_status check_species(const qed_species *s, const char *name, qed_precision prec)
{
    if (s == nullptr) QED_FAIL(QED_ERR_INVALID_ARG, "%s: species is NULL", name);
    if (prec != QED_F32 && prec != QED_F64) QED_FAIL(QED_ERR_INVALID_ARG, "%s: bad precision %d", name, (int)prec);
    const void *need[] = {s->px, s->py, s->pz, s->ex, s->ey, s->ez, s->bx, s->by, s->bz,
                          s->tau, s->weight, s->id, s->d_count};
    for (const void *p : need)
        if (p == nullptr) QED_FAIL(QED_ERR_INVALID_ARG, "%s: a species array is NULL", name);
    if (prec == QED_F32 && s->tau_c == nullptr) QED_FAIL(QED_ERR_INVALID_ARG, "%s: tau_c is required for FP32", name);
    const size_t es = prec == QED_F32 ? 4 : 8;
    const void *arrs[] = {s->px, s->py, s->pz, s->ex, s->ey, s->ez, s->bx, s->by, s->bz, s->tau, s->weight};
    for (const void *p : arrs)
        if (!aligned(p, es)) QED_FAIL(QED_ERR_INVALID_ARG, "%s: array not aligned to its element size", name);
    if (prec == QED_F32 && !aligned(s->tau_c, 4)) QED_FAIL(QED_ERR_INVALID_ARG, "%s: tau_c misaligned", name);
    if (!aligned(s->id, 8) || !aligned(s->d_count, 8)) QED_FAIL(QED_ERR_INVALID_ARG, "%s: id/d_count misaligned", name);
    if (s->capacity < 0 || s->capacity > (int64_t)1 << 40) QED_FAIL(QED_ERR_INVALID_ARG, "%s: capacity %lld out of range", name, (long long)s->capacity);
    return QED_OK;
}

// The error words of all translation units, registered during static
// initialisation (a function-local table, so the order of initialisation of
// the translation units does not matter).
struct ErrWordRegistry {
    ErrWordIO fn[64];
    int n = 0;
};

static ErrWordRegistry &err_registry()
{
    static ErrWordRegistry r;
    return r;
}

int register_err_word(ErrWordIO f)
{
    ErrWordRegistry &r = err_registry();
    if (r.n < 64) r.fn[r.n++] = f;
    return r.n;
}

}  // namespace qed

extern "C" qed_status qed_device_status(void *stream, uint32_t *word_out, int32_t clear)
{
    using namespace qed;
    clear_error();
    QED_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    unsigned w = 0;
    ErrWordRegistry &r = err_registry();
    for (int i = 0; i < r.n; ++i) {
        unsigned v = 0;
        QED_CUDA_TRY(r.fn[i](&v, clear != 0));
        w |= v;
    }
    if (word_out) *word_out = w;
    if (w & QED_EW_WAIT_TIMEOUT)
        QED_FAIL(QED_ERR_TIMEOUT, "a bounded wait gave up on the device (error word 0x%x)", w);
    if (w & (QED_EW_CAPACITY | QED_EW_FIRE_OVERFLOW))
        QED_FAIL(QED_ERR_CAPACITY, "events were left unexecuted for lack of room (error word 0x%x)", w);
    if (w & QED_EW_NONFINITE) QED_FAIL(QED_ERR_NUMERIC, "non-finite chi or optical depth seen (error word 0x%x)", w);
    return QED_OK;
}

extern "C" const char *qed_last_error_message(void) { return qed::g_err; }

extern "C" const char *qed_version(void) { return "libqed 0.1 (sm_103a)"; }
