// prof.cu -- launch counting and per-kernel CUDA-event timing.
#include <map>
#include <string>
#include <vector>

#include "api_internal.h"
#include "prof.h"

namespace mwj {

static thread_local Profiler *t_prof = nullptr;

Profiler *current_profiler() { return t_prof; }
void set_current_profiler(Profiler *p) { t_prof = p; }

ProfScope::ProfScope(const char *name, cudaStream_t s) : p(t_prof), slot(-1), st(s) {
    if (!p) return;
    p->launches++;
    if (!p->on) return;
    if (p->next + 2 > (int)p->pool.size()) return;   // pool exhausted: count only
    slot = p->next;
    p->next += 2;
    p->recs.push_back(Profiler::Rec{name, slot});
    cudaEventRecord(p->pool[slot], st);
}

ProfScope::~ProfScope() {
    if (p && slot >= 0) cudaEventRecord(p->pool[slot + 1], st);
}

void Profiler::enable(bool e, int max_launches) {
    if (e && pool.empty()) {
        pool.resize(2 * (size_t)max_launches);
        for (auto &ev : pool) cudaEventCreate(&ev);
    }
    on = e;
}

void Profiler::resolve() {
    for (const Rec &r : recs) {
        float ms = 0.f;
        cudaEventSynchronize(pool[r.slot + 1]);
        if (cudaEventElapsedTime(&ms, pool[r.slot], pool[r.slot + 1]) == cudaSuccess) {
            auto &a = acc[r.name];
            a.first += ms;
            a.second += 1;
        }
    }
    recs.clear();
    next = 0;
}

Profiler::~Profiler() {
    for (auto &ev : pool) cudaEventDestroy(ev);
}

}  // namespace mwj

namespace mwj {
ApiScope::ApiScope(Profiler *p) : prev(current_profiler()) { set_current_profiler(p); }
ApiScope::~ApiScope() { set_current_profiler(prev); }
}  // namespace mwj
