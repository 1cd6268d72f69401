// noalloc.cu -- qed_substep for callers that cannot allocate device memory.
//
// qed_substep needs three firing lists (index + chi per firing particle, and a
// count) as working memory between the evolution and the event kernels.  Some
// callers cannot provide them: codes whose device memory is entirely owned by
// their own pool allocator (a PIC framework that reserves the GPU at start-up
// and forbids foreign allocations), callers that must not trigger the implicit
// device synchronisation of cudaMalloc / cudaFree in the middle of a time step,
// and embedded runtimes that refuse new allocations after initialisation.  For
// them, qed_substep_noalloc keeps the firing lists in a fixed array compiled
// into this library, and allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoallocScratchBytes, about 16 MiB) until the process exits.
// Host code must not pass the variable's name to a kernel (on the host it is a
// stand-in, not a device address): the device address is looked up once per
// device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "common.cuh"

namespace qed {

// firing-list entries shared by the three species of one call
constexpr int64_t kNoallocMaxParticles = QED_NOALLOC_MAX_PARTICLES;
// layout: [0, 256) three int64 counts; then int64 idx[max]; then double chi[max]
constexpr size_t kNoallocHeader = 256;
constexpr size_t kNoallocScratchBytes = kNoallocHeader + (size_t)kNoallocMaxParticles * (8 + 8);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once)
static qed_status noalloc_scratch(unsigned char **out)
{
    int dev = 0;
    QED_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) QED_FAIL(QED_ERR_UNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            QED_FAIL(QED_ERR_CUDA, "cudaGetSymbolAddress of the firing-list scratch failed: %s",
                     cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = (unsigned char *)g_noalloc_ptr[dev];
    return QED_OK;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_substep_noalloc(const qed_tables *t, const qed_species *electrons,
                                          const qed_species *positrons, const qed_species *photons, double dt,
                                          uint64_t seed, int64_t step, const qed_substep_opts *opts,
                                          qed_precision prec, void *stream)
{
    clear_error();
    if (!electrons || !positrons || !photons) QED_FAIL(QED_ERR_INVALID_ARG, "a species is NULL");
    const int64_t caps[3] = {electrons->capacity, positrons->capacity, photons->capacity};
    int64_t total = 0;
    for (int64_t c : caps) {
        if (c < 0) QED_FAIL(QED_ERR_INVALID_ARG, "negative species capacity");
        if (c > kNoallocMaxParticles)  // (each one first, so that the sum cannot overflow)
            QED_FAIL(QED_ERR_INVALID_ARG,
                     "qed_substep_noalloc: a species capacity of %lld particles is more than the %lld its built-in "
                     "firing-list memory holds; use qed_substep with caller-provided firing lists",
                     (long long)c, (long long)kNoallocMaxParticles);
        total += c;
    }
    if (total > kNoallocMaxParticles)
        QED_FAIL(QED_ERR_INVALID_ARG,
                 "qed_substep_noalloc: the three species' capacities add up to %lld particles, more than the "
                 "%lld its built-in firing-list memory holds; use qed_substep with caller-provided firing lists",
                 (long long)total, (long long)kNoallocMaxParticles);
    unsigned char *base = nullptr;
    qed_status s = noalloc_scratch(&base);
    if (s) return s;
    int64_t *counts = (int64_t *)base;
    int64_t *idx = (int64_t *)(base + kNoallocHeader);
    double *chi = (double *)(base + kNoallocHeader + (size_t)kNoallocMaxParticles * 8);
    // each species gets a slice as long as its capacity; qed_substep zeroes the
    // three counts on the stream before its evolution kernel writes them
    qed_fire_list fire[3];
    int64_t off = 0;
    for (int k = 0; k < 3; ++k) {
        fire[k].idx = idx + off;
        fire[k].chi = chi + off;
        fire[k].d_count = counts + k;
        fire[k].capacity = caps[k];
        off += caps[k];
    }
    return qed_substep(t, electrons, positrons, photons, dt, seed, step, opts, prec, fire, stream);
}
