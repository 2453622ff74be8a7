// prof.cu -- optional per-kernel timing with CUDA events (process-wide).
#include <mutex>
#include <vector>

#include "prof.cuh"

namespace rfm {

namespace {
struct Rec {
    const char *name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
std::vector<Rec> g_recs;
bool g_on = false;
}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t st) : name_(name), st_(st), on_(false) {
    if (!g_on) return;
    if (cudaEventCreate((cudaEvent_t *)&a_) != cudaSuccess) return;
    if (cudaEventCreate((cudaEvent_t *)&b_) != cudaSuccess) {
        cudaEventDestroy((cudaEvent_t)a_);
        return;
    }
    cudaEventRecord((cudaEvent_t)a_, st_);
    on_ = true;
}

ProfScope::~ProfScope() {
    if (!on_) return;
    cudaEventRecord((cudaEvent_t)b_, st_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back(Rec{name_, (cudaEvent_t)a_, (cudaEvent_t)b_});
}

void prof_enable(bool on) { g_on = on; }

void prof_reset() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
}

int prof_read(const char **names, int64_t *launches, double *ms, int max) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<const char *> nm;
    std::vector<int64_t> cnt;
    std::vector<double> tot;
    for (auto &r : g_recs) {
        cudaEventSynchronize(r.b);
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        size_t i = 0;
        for (; i < nm.size(); ++i)
            if (nm[i] == r.name) break;
        if (i == nm.size()) {
            nm.push_back(r.name);
            cnt.push_back(0);
            tot.push_back(0.0);
        }
        cnt[i] += 1;
        tot[i] += t;
    }
    int n = (int)nm.size();
    for (int i = 0; i < n && i < max; ++i) {
        if (names) names[i] = nm[i];
        if (launches) launches[i] = cnt[i];
        if (ms) ms[i] = tot[i];
    }
    return n;
}

}  // namespace rfm
