// The CPU side of the GPU + CPU race (MCS_RACE), see mcs_cpu.cpp.
#pragma once
#include <cstdint>

struct CpuRaceResult {
    int size;                 // best mapping found
    uint64_t nodes;           // search nodes expanded
    bool complete;            // the search finished: its size (with the GPU's) is proven
    int16_t g[64], h[64];     // the mapping, original vertex numbers
};

// Sequential McSplit of one pair of graphs of at most 64 vertices (layout of
// mcs_graph), pruning against max(own best, *gpu_best); publishes its best
// size in *cpu_best; stops early when *stop becomes nonzero or at timeout_s
// (<= 0: none).  Returns 0, or -1 for malformed input.
int cpu_mcs_race(int nG, const uint8_t* adjG, const int32_t* labG, int nH, const uint8_t* adjH,
                 const int32_t* labH, bool directed, double timeout_s, const volatile int32_t* gpu_best,
                 volatile int32_t* cpu_best, const volatile int32_t* stop, CpuRaceResult* out);
