// Round trip of the autotune cache file (tune_cache_store / tune_cache_lookup of pfc_host.h;
// host code only, compiled by tests/test_planner.py).
//   tune_cache PATH   appends three entries for two keys, then prints one JSON object per
//                     lookup: {"key": .., "found": .., "Py": .., "Pz": .., "W": .., "cluster": .., "ms": ..}
#include <cstdio>

#include "../../paper_2603_26818_gb300/csrc/pfc_host.h"

static void show(const char *path, const char *key) {
    pfc::TileChoice c;
    double ms = -1;
    const bool found = pfc::tune_cache_lookup(path, key, c, ms);
    std::printf("{\"key\": \"%s\", \"found\": %s, \"Py\": %d, \"Pz\": %d, \"W\": %d, \"cluster\": %d, \"ms\": %.6f}\n",
                key, found ? "true" : "false", c.Py, c.Pz, c.W, c.cluster, ms);
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    const char *path = argv[1];
    pfc::TileChoice a;
    a.Py = 8; a.Pz = 1; a.W = 4; a.cluster = 1;
    pfc::TileChoice b;
    b.Py = 2; b.Pz = 2; b.W = 8; b.cluster = 0;
    pfc::TileChoice a2 = a;
    a2.W = 2;
    pfc::tune_cache_store(path, "1x4096x4096 prec1 fields1 NVIDIA_GB300", a, 0.158475);
    pfc::tune_cache_store(path, "256x256x256 prec1 fields2 NVIDIA_GB300", b, 0.556376);
    pfc::tune_cache_store(path, "1x4096x4096 prec1 fields1 NVIDIA_GB300", a2, 0.16);
    show(path, "1x4096x4096 prec1 fields1 NVIDIA_GB300");
    show(path, "256x256x256 prec1 fields2 NVIDIA_GB300");
    show(path, "512x512x512 prec1 fields1 NVIDIA_GB300");
    return 0;
}
