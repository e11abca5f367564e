// Internal declarations shared by the library's host driver and kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fpsa.h"

namespace fpsa {

// S_N tables (host, FP64). Matrices row-major N x N; moments padded to N.
struct Tables {
    int N = 0, L1 = 0;
    std::vector<double> mu, w;
    std::vector<double> D;    // D[l][n] = w_n P_l(mu_n)
    std::vector<double> M;    // M[n][l] = (2l+1)/2 P_l(mu_n), zero for l >= L1
    std::vector<double> Afp;  // discrete angular Laplacian (MPD or WFD)
};
void build_tables(int N, int L1, int laplacian, Tables &t);

// One cell eliminated at one block-cyclic-reduction level (or an instance root).
// Cell ids are global (concatenated over instances); -1 = absent.
// Coupling slots index the per-level N/2 x N/2 coupling blocks B (to the left
// neighbour's right-node mu>0 values) and C (to the right neighbour's left-node
// mu<0 values): slot(j, l) = slot_base[j] + l.
struct BcrItem {
    int32_t cell, left, right;
    int32_t s_cell;        // slot(cell, l)
    int32_t s_left;        // slot(left, l)
    int32_t s_left_next;   // slot(left, l+1)
    int32_t s_right;       // slot(right, l)
    int32_t s_right_next;  // slot(right, l+1)
    int32_t local;         // cell index within its instance
    int32_t K_inst;        // cells of the instance
    int32_t level;         // level the cell is eliminated at (roots: the instance's level count)
};

// Device-side geometry of the batch.
struct Geometry {
    int B = 0, N = 0, L1 = 0, R = 0, sumK = 0, Kmax = 0;
    int n_levels = 0;                   // max over instances
    int n_slots = 0;
    std::vector<int32_t> K, off;        // per instance
    std::vector<int32_t> cell_inst;     // per global cell
    std::vector<int32_t> slot_base;     // per global cell
    std::vector<std::vector<BcrItem>> levels;  // [level] -> items over all instances
    std::vector<BcrItem> roots;         // one per instance
};
void build_geometry(const int32_t *K, int B, int N, int L1, int R, Geometry &g);

}  // namespace fpsa
