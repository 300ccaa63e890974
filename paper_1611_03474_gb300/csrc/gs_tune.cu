// gs_tune.cu -- launch-shape autotuner.
//
// A kernel with several launch shapes that compute the same result (tile
// shape, grid size) is launched through gs_tune_run.  The first launch for a
// (kernel, size class) pair times every shape on the call's own data -- one
// untimed and two timed launches each, CUDA events on the call's stream,
// counters sent to a scratch buffer -- keeps the fastest, and then launches
// it for real; later launches of that class take the recorded choice.  Size
// classes are powers of two of the item count.  The choices, with the
// trial times, are listed by gs_autotune_report.
//
// GS_AUTOTUNE=0 (environment) turns tuning off: every launch takes shape 0,
// the default; GS_AUTOTUNE=shape:K takes shape K (the last one where a
// kernel has fewer), for tests that compare the shapes.  A stream under
// graph capture takes the recorded choice or shape 0 (a trial would
// synchronise inside the capture).
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gs_host.cuh"

namespace {
struct TuneEntry {
    int choice = 0;
    std::vector<float> ms;
};
std::mutex g_tune_mu;
std::map<std::pair<std::string, int>, TuneEntry> g_tune;

int size_class(int64_t n)
{
    int k = 0;
    while (k < 62 && ((int64_t)1 << (k + 1)) <= n) k++;
    return k;
}

// -1: tune; else the shape to take without tuning
int forced_shape(int n_choices)
{
    const char *s = getenv("GS_AUTOTUNE");
    if (!s) return -1;
    if (!strcmp(s, "0")) return 0;
    if (!strncmp(s, "shape:", 6)) {
        const int k = atoi(s + 6);
        return k < 0 ? 0 : (k >= n_choices ? n_choices - 1 : k);
    }
    return -1;
}
}  // namespace

int gs_tune_run(const char *kernel, int64_t n, int n_choices, cudaStream_t st,
                const std::function<void(int, unsigned long long *)> &launch)
{
    const int forced = forced_shape(n_choices);
    if (forced >= 0) {
        launch(forced, nullptr);
        GS_CHECK(cudaGetLastError());
        return GS_OK;
    }
    const auto key = std::make_pair(std::string(kernel), size_class(n));
    int choice = 0;
    bool found = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) { choice = it->second.choice; found = true; }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!found && n_choices > 1 && cudaStreamIsCapturing(st, &cap) == cudaSuccess &&
        cap == cudaStreamCaptureStatusNone) {
        unsigned long long *scratch = nullptr;
        int rc = gs_alloc((void **)&scratch, 32 * sizeof(unsigned long long), st);
        if (rc) return rc;
        cudaEvent_t e0, e1;
        GS_CHECK(cudaEventCreate(&e0));
        GS_CHECK(cudaEventCreate(&e1));
        TuneEntry ent;
        ent.ms.assign((size_t)n_choices, 0.f);
        cudaError_t e = cudaSuccess;
        for (int c = 0; c < n_choices && e == cudaSuccess; c++) {
            launch(c, scratch);   // untimed: module load, caches
            float best = 3.4e38f;
            for (int r = 0; r < 2 && e == cudaSuccess; r++) {
                cudaEventRecord(e0, st);
                launch(c, scratch);
                cudaEventRecord(e1, st);
                e = cudaEventSynchronize(e1);
                float t = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (t < best) best = t;
            }
            if (e == cudaSuccess) e = cudaGetLastError();
            ent.ms[(size_t)c] = best;
            if (best < ent.ms[(size_t)ent.choice]) ent.choice = c;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        gs_free(scratch, st);
        if (e != cudaSuccess) return gs_fail_cuda(e, "autotune trial", __FILE__, __LINE__);
        choice = ent.choice;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = ent;
    }
    launch(choice, nullptr);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

extern "C" int64_t gs_autotune_report(char *buf, int64_t cap)
{
    std::string s;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto &kv : g_tune) {
            char line[256];
            int k = snprintf(line, sizeof(line), "%s 2^%d %d", kv.first.first.c_str(), kv.first.second,
                             kv.second.choice);
            std::string l(line, (size_t)(k > 0 ? k : 0));
            for (float t : kv.second.ms) {
                snprintf(line, sizeof(line), " %.4f", t);
                l += line;
            }
            s += l + "\n";
        }
    }
    if (buf && cap > 0) {
        const size_t m = s.size() < (size_t)(cap - 1) ? s.size() : (size_t)(cap - 1);
        memcpy(buf, s.data(), m);
        buf[m] = 0;
    }
    return (int64_t)s.size() + 1;
}

extern "C" void gs_autotune_reset(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}
