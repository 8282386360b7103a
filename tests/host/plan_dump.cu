// Prints the tile plan chosen by plan_tiles for every shape given on the command line, one JSON
// object per line (host code only; compiled by tests/test_planner.py).
//   plan_dump NX NY NZ VB NTILE INSTANCES [NX NY NZ VB NTILE INSTANCES ...]
// With PLAN_DUMP_ALL set it prints instead every candidate tiling the autotuner may time
// (tile_candidates, each with the clustered row pass on and, where it applies, off), with its
// rank in "cand"; PLAN_DUMP_SCHED=3 lists the three-pass candidates instead.
#include <cstdio>
#include <cstdlib>

#include "../../paper_2603_26818_gb300/csrc/pfc_host.h"

static void print_plan(const pfc::Tiles &t, int nx, int ny, int nz, size_t vb, int ntile, int inst, int cand) {
    const pfc::Geom &g = t.g;
    std::printf("{\"nx\": %d, \"ny\": %d, \"nz\": %d, \"vb\": %zu, \"ntile\": %d, \"ok\": true, \"M\": %d, "
                "\"Py\": %d, \"Pz\": %d, \"Qy\": %d, \"Qz\": %d, \"P\": %d, \"Q\": %d, \"W\": %d, \"xs\": %d, "
                "\"ncg\": %d, \"tsz\": %d, \"rs\": %d, \"gpc\": %d, \"nt_row\": %d, \"nt_line\": %d, "
                "\"smem_row\": %zu, \"smem_line\": %zu, \"row_cs\": %d, \"nt_row_cs\": %d, "
                "\"smem_row_cs\": %zu, \"nhalf\": %lld, \"inst\": %d, \"cand\": %d, \"Ry\": %d, \"Rz\": %d, "
                "\"R\": %d, \"QR\": %d}\n",
                nx, ny, nz, vb, ntile, g.M, g.Py, g.Pz, g.Qy, g.Qz, g.P, g.Q, g.W, g.xs, g.ncg, g.tsz, g.rs,
                g.gpc, t.nt_row, t.nt_line, t.smem_row, t.smem_line, t.row_cs, t.nt_row_cs, t.smem_row_cs,
                (long long)g.nhalf, inst, cand, g.Ry, g.Rz, g.R, g.QR);
}

int main(int argc, char **argv) {
    const size_t smem_max = 232448;   // sm_103a opt-in shared memory per block
    for (int i = 1; i + 5 < argc; i += 6) {
        const int nx = std::atoi(argv[i]), ny = std::atoi(argv[i + 1]), nz = std::atoi(argv[i + 2]);
        const size_t vb = (size_t)std::atoi(argv[i + 3]);
        const int ntile = std::atoi(argv[i + 4]), inst = std::atoi(argv[i + 5]);
        if (std::getenv("PLAN_DUMP_ALL")) {
            int rank = 0;
            const char *sc = std::getenv("PLAN_DUMP_SCHED");
            const int sched = sc ? std::atoi(sc) : pfc::SCHED_AUTO;
            for (const pfc::TileChoice &c0 :
                 pfc::tile_candidates(nx, ny, nz, vb, ntile, smem_max, pfc::TileChoice{}, inst, sched)) {
                for (int cl = 1; cl >= 0; --cl) {
                    pfc::TileChoice c = c0;
                    c.cluster = cl;
                    pfc::Tiles t;
                    if (!pfc::plan_tiles_as(t, c, nx, ny, nz, vb, ntile, smem_max, inst)) {
                        std::printf("{\"nx\": %d, \"ny\": %d, \"nz\": %d, \"vb\": %zu, \"ok\": false, \"cand\": %d}\n",
                                    nx, ny, nz, vb, rank);
                        break;
                    }
                    print_plan(t, nx, ny, nz, vb, ntile, inst, rank);
                    if (t.row_cs == 0) break;
                }
                ++rank;
            }
            continue;
        }
        pfc::Tiles t;
        if (!pfc::plan_tiles(t, nx, ny, nz, vb, ntile, smem_max, inst)) {
            std::printf("{\"nx\": %d, \"ny\": %d, \"nz\": %d, \"vb\": %zu, \"ok\": false}\n", nx, ny, nz, vb);
            continue;
        }
        print_plan(t, nx, ny, nz, vb, ntile, inst, -1);
    }
    return 0;
}
