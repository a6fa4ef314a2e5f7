// nb_force_static: a force evaluation that allocates no memory at all.
//
// Some callers cannot call cudaMalloc. A host code that hands all of its
// device memory to its own pool allocator (a tree code coupled to this
// library, for instance) may forbid any other allocation, since cudaMalloc
// synchronises the device and fragments the pool; other callers run where
// no allocation is allowed at all. Those callers pass their own device
// buffers for inputs and outputs; the only scratch this call needs, the
// partial sums of its j-split, lives in the fixed array below.
//
// The array is a file-scope __device__ variable (8 MiB). CUDA loads a
// library's device code lazily, so the array, and the force kernels this call
// launches, take their device memory when they are first used on a device,
// not when the library is loaded; from then on the device holds them until the
// process exits. Host code cannot use the symbol itself as a device address,
// so the first call on each device (with that device current) looks the
// address up with cudaGetSymbolAddress, caches it, and loads and runs the
// kernels once on an empty i-set. That first call is the per-device warm-up:
// a caller whose pool allocator will own the device memory makes it, with
// n_i = 0, before the pool takes the memory, and no later call allocates.
#include <cuda_runtime.h>

#include <mutex>

#include "nb_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;

// Partial sums of the j-split: 7 values per (split, i-particle).
__device__ __align__(256) double g_static_part[NB_STATIC_SCRATCH_DOUBLES];
// Device error word of these calls (cleared at the start of every call), and
// the arrival counter of the split reduction (re-armed to zero by each call).
__device__ __align__(256) unsigned g_static_err[64];
__device__ __align__(256) unsigned g_static_cnt[64];

struct StaticSlot {
    double *part = nullptr;
    unsigned *err = nullptr;
    unsigned *cnt = nullptr;
    int num_sms = 0;
    bool ready = false;
};

StaticSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;

// Per-device set-up: the device addresses of the static arrays (which loads
// this file's device code), then the force kernels loaded and run once.
int static_slot(int dev, cudaStream_t st, StaticSlot *out)
{
    std::lock_guard<std::mutex> lk(g_slots_mu);
    StaticSlot &s = g_slots[dev];
    if (!s.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_part) != cudaSuccess) {
            cudaGetLastError();
            return NB_ERR_CUDA;
        }
        s.part = static_cast<double *>(p);
        if (cudaGetSymbolAddress(&p, g_static_err) != cudaSuccess) {
            cudaGetLastError();
            return NB_ERR_CUDA;
        }
        s.err = static_cast<unsigned *>(p);
        if (cudaGetSymbolAddress(&p, g_static_cnt) != cudaSuccess) {
            cudaGetLastError();
            return NB_ERR_CUDA;
        }
        s.cnt = static_cast<unsigned *>(p);
        if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess) {
            cudaGetLastError();
            return NB_ERR_CUDA;
        }
        if (nb::warm_force_jmode64(st) != cudaSuccess ||
            cudaMemsetAsync(s.err, 0, sizeof(unsigned), st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return NB_ERR_CUDA;
        }
        s.ready = true;
    }
    *out = s;
    return NB_OK;
}

}  // namespace

extern "C" int nb_force_static(int n_j, const double *m, const double *pos, const double *vel,
                               long long ld, int n_i, const int *idx, double eps, double *acc,
                               double *jerk, double *pot, void *stream)
{
    if (n_j < 1 || !m || !pos || !vel || ld < n_j) return NB_ERR_ARG;
    if (n_i < 0 || n_i > NB_STATIC_MAX_NI) return NB_ERR_ARG;
    if (!idx && n_i > n_j) return NB_ERR_ARG;
    if (!(eps >= 0.0) || eps != eps) return NB_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StaticSlot slot;
    int rc = static_slot(dev, st, &slot);  // the warm-up, on the first call on this device
    if (rc) return rc;
    if (n_i == 0) return NB_OK;

    nb::JSet js{};
    js.n = n_j;
    js.rec32 = nullptr;
    js.pos64 = pos;
    js.vel64 = vel;
    js.m64 = m;
    js.ld = ld;
    nb::ISet is{};
    is.n = n_i;
    is.idx = idx;
    is.member = true;
    is.rec32 = nullptr;
    is.pos64 = pos;
    is.vel64 = vel;
    is.m64 = m;
    is.ld64 = ld;
    is.nj = n_j;
    is.gathered = false;

    // FP64 j-parallel plan whose partial sums fit the static array.
    nb::ForcePlan plan{};
    plan.kind = 1;
    plan.threads = 128;
    plan.ipt = n_i <= 1 ? 1 : (n_i <= 2 ? 2 : 4);
    long long ns = ((long long)n_j + 128 * 4 - 1) / (128 * 4);
    if (ns > 2LL * slot.num_sms) ns = 2LL * slot.num_sms;
    const long long fit = NB_STATIC_SCRATCH_DOUBLES / (7LL * n_i);
    if (ns > fit) ns = fit;
    if (ns < 1) ns = 1;
    plan.nsplit = (int)ns;
    plan.jt = 0;

    if (cudaMemsetAsync(slot.err, 0, sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(slot.cnt, 0, sizeof(unsigned), st) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    nb::Out3 out{acc, jerk, pot, n_i};
    if (nb::launch_force(NB_F64, plan, js, is, eps * eps, slot.part, slot.cnt, out, slot.err, st,
                         nullptr) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, slot.err, sizeof e, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    if (e & nb::DERR_BADINDEX) return NB_ERR_ARG;
    if (e & nb::DERR_TIMEOUT) return NB_ERR_TIMEOUT;
    if (e) return NB_ERR_NONFINITE;
    return NB_OK;
}
