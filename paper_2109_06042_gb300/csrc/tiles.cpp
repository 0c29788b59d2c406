// tiles.cpp -- the tile shape of the tcgen05 contraction: explicit options,
// or the autotuner's table.
//
// The shape of a launch is three choices that change no result, only speed:
// the tile width (128 x 256 tiles with two TMEM accumulators, or 128 x 128
// with four), the row blocks per L2 group of the tile order, and whether a
// K block shared in one half only is loaded as that half.  Options left at
// 0 are looked up in a table written by the autotuner
// (paper_2109_06042_gb300/autotune.py), which times every shape on seeded
// workloads of each size class on the GPU and keeps the fastest.  The table
// is the text file named by the environment variable MHS_TILE_TABLE, or
// tile_table.txt beside this library.  One line per size class:
//     <kind> <log2 rows> <tile_n> <group_rows> <half_stages>
// kind is "single" (one instance) or "batch"; log2 rows is floor(log2) of
// the larger of n and m (a batch: its mean over the instances).  A class
// missing from the table takes the nearest class of the same kind; with no
// table at all, the defaults (256, 16 or MHS_TILE_GROUP_ROWS, halves on).
#include <dlfcn.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "host_internal.h"
#include "kernels.h"

namespace mhs {
namespace {

struct Entry {
    int kind;  // 0 single, 1 batch
    int log2rows;
    int32_t tile_n, group_rows, half_stages;
};

std::once_flag g_once;
std::vector<Entry> g_table;
std::string g_table_path;

std::string library_dir() {
    Dl_info info;
    if (dladdr(reinterpret_cast<void *>(&library_dir), &info) && info.dli_fname) {
        std::string p = info.dli_fname;
        const size_t k = p.rfind('/');
        return k == std::string::npos ? std::string(".") : p.substr(0, k);
    }
    return ".";
}

void load_table() {
    const char *env = std::getenv("MHS_TILE_TABLE");
    g_table_path = env && *env ? std::string(env) : library_dir() + "/tile_table.txt";
    FILE *fh = std::fopen(g_table_path.c_str(), "r");
    if (!fh) return;
    char line[512];
    while (std::fgets(line, sizeof(line), fh)) {
        char *hash = std::strchr(line, '#');
        if (hash) *hash = '\0';
        char kind[32];
        int lg = 0, tn = 0, gr = 0, hs = 0;
        if (std::sscanf(line, "%31s %d %d %d %d", kind, &lg, &tn, &gr, &hs) != 5) continue;
        const int k = std::strcmp(kind, "single") == 0 ? 0 : std::strcmp(kind, "batch") == 0 ? 1 : -1;
        if (k < 0 || (tn != 128 && tn != 256) || gr < 1 || gr > 4096 || hs < 1 || hs > 2 || lg < 0 ||
            lg > 31)
            continue;  // a malformed line is skipped, never half applied
        g_table.push_back({k, lg, tn, gr, hs});
    }
    std::fclose(fh);
}

int floor_log2(int64_t x) {
    int l = 0;
    while (x > 1) { x >>= 1; ++l; }
    return l;
}

}  // namespace

TileChoice choose_tiles(int32_t count, int64_t typical_rows, const mhs_options &opt) {
    std::call_once(g_once, load_table);
    TileChoice c;
    c.tile_n = kTcNDefault;
    c.group_rows = tile_group_rows();
    c.half_stages = 1;
    c.from_table = 0;
    const int kind = count > 1 ? 1 : 0;
    const int lg = floor_log2(typical_rows > 0 ? typical_rows : 1);
    const Entry *best = nullptr;
    for (const Entry &e : g_table) {
        if (e.kind != kind) continue;
        if (!best || std::abs(e.log2rows - lg) < std::abs(best->log2rows - lg)) best = &e;
    }
    if (best) {
        c.tile_n = best->tile_n;
        c.group_rows = best->group_rows;
        c.half_stages = best->half_stages == 1 ? 1 : 0;
        c.from_table = 1;
    }
    // explicit options win over the table; from_table says whether the table
    // gave any of the three
    if (opt.tile_n) c.tile_n = opt.tile_n;
    if (opt.group_rows) c.group_rows = opt.group_rows;
    if (opt.half_stages) c.half_stages = opt.half_stages == 1 ? 1 : 0;
    if (opt.tile_n && opt.group_rows && opt.half_stages) c.from_table = 0;
    return c;
}

const char *tile_table_path() {
    std::call_once(g_once, load_table);
    return g_table_path.c_str();
}

}  // namespace mhs
