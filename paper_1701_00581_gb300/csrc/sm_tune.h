// Shape of the batched persistent launch per (N, R).  Written by
// paper_1701_00581_gb300/autotune.py from timings of the launch on the GPU;
// the library picks the entry of the batch's largest N with the nearest R.
#pragma once

namespace smt {

struct TuneEntry {
    int N, R;
    int lookahead, ctas_per_sm, launch, tile_order;
    double ms_per_burst;          // the winning configuration's launch time per burst (0: not measured)
};

// BEGIN TABLE (autotune.py)
constexpr TuneEntry kTune[] = {
    {256, 24, 2, 4, 3, 1, 110.051},
    {128, 16, 2, 4, 3, 1, 14.249},
    {64, 8, 2, 4, 3, 1, 0.021},
};
// END TABLE

inline TuneEntry tune_for(int N, int R) {
    const TuneEntry* best = nullptr;
    for (const TuneEntry& e : kTune) {
        if (e.N != N) continue;
        if (!best || (e.R > R ? e.R - R : R - e.R) < (best->R > R ? best->R - R : R - best->R)) best = &e;
    }
    if (!best)
        for (const TuneEntry& e : kTune)
            if (!best || (e.N > N ? e.N - N : N - e.N) < (best->N > N ? best->N - N : N - best->N)) best = &e;
    return *best;
}

}  // namespace smt
