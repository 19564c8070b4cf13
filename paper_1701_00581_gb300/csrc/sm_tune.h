// Shape of the batched launch per (N, R) and launch kind: the fastest
// lookahead, CTAs per SM and tile order for each of the three launches.
// Written by paper_1701_00581_gb300/autotune.py from timings of the launch
// on the GPU.
#pragma once

namespace smt {

struct TuneEntry {
    int N, R;
    int lookahead, ctas_per_sm, launch, tile_order;
    double ms_per_burst;          // the winning configuration's launch time per burst (0: not measured)
};

// BEGIN TABLE (autotune.py)
constexpr TuneEntry kTune[] = {
    {256, 24, 4, 4, 1, 1, 109.7350},
    {256, 24, 2, 4, 2, 1, 108.4027},
    {256, 24, 2, 4, 3, 1, 108.5971},
    {128, 16, 4, 4, 1, 2, 14.0166},
    {128, 16, 2, 4, 2, 2, 14.2122},
    {128, 16, 2, 4, 3, 1, 14.1201},
    {64, 8, 4, 3, 1, 1, 0.0238},
    {64, 8, 2, 3, 2, 2, 0.0218},
    {64, 8, 2, 4, 3, 1, 0.0209},
};
// END TABLE

// The entry for a batch: the table's (N, R) nearest to the batch's largest
// subfield size N (the same N if the table has it) and then its R; among
// that shape's entries, the one for the requested launch shape, or the
// fastest when the launch is left to the table (launch = 0).
inline TuneEntry tune_for(int N, int R, int launch) {
    auto dist = [](int a, int b) { return a > b ? a - b : b - a; };
    int bn = -1, br = -1;
    for (const TuneEntry& e : kTune) {
        if (bn < 0 || dist(e.N, N) < dist(bn, N) || (e.N == bn && dist(e.R, R) < dist(br, R))) {
            bn = e.N;
            br = e.R;
        }
    }
    const TuneEntry* best = nullptr;
    for (const TuneEntry& e : kTune) {
        if (e.N != bn || e.R != br) continue;
        if (launch != 0 && e.launch != launch) continue;
        if (!best || e.ms_per_burst < best->ms_per_burst) best = &e;
    }
    if (!best)                                       // the shape has no entry for that launch
        for (const TuneEntry& e : kTune)
            if (e.N == bn && e.R == br && (!best || e.ms_per_burst < best->ms_per_burst)) best = &e;
    TuneEntry t = *best;
    if (launch != 0) t.launch = launch;
    return t;
}

}  // namespace smt
