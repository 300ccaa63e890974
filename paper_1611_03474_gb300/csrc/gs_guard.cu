// gs_guard.cu -- host waits with a deadline, and host-side fault injection
// for testing the library's error paths without faulting the GPU.
//
// gs_sync(st) replaces cudaStreamSynchronize for every host wait of the
// library: it records an event on the stream and polls it (a short spin,
// then sleeps of 20 us) until the work is done, a CUDA error comes back, or
// the deadline passes (GS_WAIT_TIMEOUT_S seconds, default 600), in which case
// it returns cudaErrorTimeout and the call returns GS_ERR_TIMEOUT.  Every
// device loop of the library is bounded, so the deadline only guards
// against a stalled device or a neighbour that holds it.
//
// GS_FAULT (environment, read at each API call; injection is host-side
// only and never touches the device):
//   alloc@K     the K-th device allocation of the call fails (GS_ERR_OOM)
//   capacity@L  the level loop reports a full internal table at level L on
//               the call's first attempt (the call retries with smaller
//               level chunks, as for a real overflow)
//   timeout     the call's first host wait times out (GS_ERR_TIMEOUT)
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <thread>

#include "gs_host.cuh"

namespace {
enum FaultKind { F_NONE = 0, F_ALLOC = 1, F_CAPACITY = 2, F_TIMEOUT = 3 };
struct FaultState {
    int kind = F_NONE;
    long long arg = 0;
    long long allocs = 0;
    bool fired = false;
};
thread_local FaultState g_fault;
}  // namespace

void gs_guard_begin(void)
{
    g_fault = FaultState();
    const char *s = getenv("GS_FAULT");
    if (!s || !*s) return;
    if (!strncmp(s, "alloc@", 6)) {
        g_fault.kind = F_ALLOC;
        g_fault.arg = atoll(s + 6);
    } else if (!strncmp(s, "capacity@", 9)) {
        g_fault.kind = F_CAPACITY;
        g_fault.arg = atoll(s + 9);
    } else if (!strcmp(s, "timeout")) {
        g_fault.kind = F_TIMEOUT;
    }
}

bool gs_fault_alloc(void)
{
    if (g_fault.kind != F_ALLOC || g_fault.fired) return false;
    if (++g_fault.allocs < g_fault.arg) return false;
    g_fault.fired = true;
    return true;
}

bool gs_fault_capacity(int level)
{
    if (g_fault.kind != F_CAPACITY || g_fault.fired || level != g_fault.arg) return false;
    g_fault.fired = true;
    return true;
}

static double wait_limit_s(void)
{
    const char *s = getenv("GS_WAIT_TIMEOUT_S");
    double v = s ? atof(s) : 0.0;
    return v > 0.0 ? v : 600.0;
}

cudaError_t gs_sync(cudaStream_t st)
{
    if (g_fault.kind == F_TIMEOUT && !g_fault.fired) {
        g_fault.fired = true;
        cudaStreamSynchronize(st);   // leave nothing in flight behind the injected failure
        return cudaErrorTimeout;
    }
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, st);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return e;
    }
    const auto t0 = std::chrono::steady_clock::now();
    const double limit = wait_limit_s();
    for (long long it = 0;; it++) {
        e = cudaEventQuery(ev);
        if (e != cudaErrorNotReady) break;
        if (it > 64) {
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (dt > limit) {
                e = cudaErrorTimeout;
                break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    cudaEventDestroy(ev);
    return e;
}
