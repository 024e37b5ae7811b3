// prof.h -- the profiler object held by a context.
#pragma once

#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace mwj {

struct Profiler {
    struct Rec {
        const char *name;
        int slot;
    };
    bool on = false;
    long long launches = 0;
    int next = 0;
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    std::map<std::string, std::pair<double, long long>> acc;   // name -> (ms, launches)
    void enable(bool e, int max_launches);
    void resolve();
    ~Profiler();
};

// Makes `p` the profiler of the launches issued on this thread until the
// scope ends (set at every C-ABI entry point).
struct ApiScope {
    Profiler *prev;
    explicit ApiScope(Profiler *p);
    ~ApiScope();
};

}  // namespace mwj
