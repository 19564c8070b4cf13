// Host-side plan object and helpers shared by the plan builder and the API.
#pragma once

#include <string>
#include <vector>

#include "sm_internal.h"

struct sm_plan {
    sm_channel ch;
    int device = 0;
    smi::PlanDev dev;
    std::vector<int4> subs;
    std::vector<int4> tiles;
    std::vector<unsigned> tile_masks;   // [tile] byte q: offset columns of row q holding a used pair
    std::vector<int> tile_of;        // [w-block][v-block] -> tile id or -1
    int n_vbx = 0, n_vby = 0;
    std::vector<int> wb_start, wb_tiles;
    std::vector<int> ring_start;
    std::vector<int2> points;
    std::vector<int4> items;
    std::vector<int> ring_items, point_items;
    std::vector<int4> point_rec;
    std::vector<int> cubes, cube_of_sub;   // seeing cubes (subfield ids), subfield -> cube or -1
    std::vector<int> ann_start, ann_idx;   // annuli of the half-plane domain
    std::vector<int> ref_start, ref_idx;   // refinement partial slots of each recursion point
    long long n_pairs = 0;
    int n_U = 0, n_V = 0;
    void* dmem = nullptr;            // device copy of every table
};

namespace smi {
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
int validate_channel(const sm_channel* ch);
bool pair_used_host(int wx, int wy, int vx, int vy, int r2i, int R2);
extern thread_local std::string g_last_error;
}  // namespace smi
