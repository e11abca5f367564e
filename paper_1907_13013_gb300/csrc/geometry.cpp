// Batch geometry and the block-cyclic-reduction schedule (host side).
//
// Instance b with K_b cells is reduced in ceil(log2 K_b) levels: level l
// eliminates the local cells i = 2^l (2k+1) < K_b, whose neighbours at that
// level are i -/+ 2^l; cell 0 is the root solved last. Every cell keeps one
// N/2 x N/2 coupling slot per level it is active in (B and C buffers share the
// slot numbering): cell i > 0 is active at levels 0..ctz(i), cell 0 at
// levels 0..n_levels(b) (one spare slot so a kept cell can always write its
// next-level coupling).
#include "fpsa_internal.h"

namespace fpsa {

static int levels_for(int K) {
    int l = 0;
    while ((1 << l) < K) ++l;
    return l;
}

static int ctz(int x) {
    int t = 0;
    while (!(x & 1)) { x >>= 1; ++t; }
    return t;
}

void build_geometry(const int32_t *K, int B, int N, int L1, int R, Geometry &g) {
    g.B = B; g.N = N; g.L1 = L1; g.R = R;
    g.K.assign(K, K + B);
    g.off.assign(B, 0);
    g.sumK = 0;
    g.Kmax = 0;
    g.n_levels = 0;
    for (int b = 0; b < B; ++b) {
        g.off[b] = g.sumK;
        g.sumK += K[b];
        if (K[b] > g.Kmax) g.Kmax = K[b];
        int nl = levels_for(K[b]);
        if (nl > g.n_levels) g.n_levels = nl;
    }
    g.cell_inst.assign(g.sumK, 0);
    g.slot_base.assign(g.sumK, 0);
    int s = 0;
    for (int b = 0; b < B; ++b) {
        int nl = levels_for(K[b]);
        for (int i = 0; i < K[b]; ++i) {
            int gc = g.off[b] + i;
            g.cell_inst[gc] = b;
            g.slot_base[gc] = s;
            s += (i == 0) ? nl + 1 : ctz(i) + 1;
        }
    }
    g.n_slots = s;
    g.levels.assign(g.n_levels, {});
    for (int l = 0; l < g.n_levels; ++l) {
        const int st = 1 << l;
        for (int b = 0; b < B; ++b) {
            for (int i = st; i < K[b]; i += 2 * st) {
                BcrItem it;
                it.cell = g.off[b] + i;
                it.left = it.cell - st;
                it.right = (i + st < K[b]) ? it.cell + st : -1;
                it.s_cell = g.slot_base[it.cell] + l;
                it.s_left = g.slot_base[it.left] + l;
                it.s_left_next = g.slot_base[it.left] + l + 1;
                it.s_right = it.right >= 0 ? g.slot_base[it.right] + l : -1;
                it.s_right_next = it.right >= 0 ? g.slot_base[it.right] + l + 1 : -1;
                it.local = i;
                it.K_inst = K[b];
                it.level = l;
                g.levels[l].push_back(it);
            }
        }
    }
    g.roots.clear();
    for (int b = 0; b < B; ++b) {
        BcrItem it{};
        it.cell = g.off[b];
        it.left = it.right = -1;
        it.s_cell = g.slot_base[it.cell] + levels_for(K[b]);
        it.s_left = it.s_left_next = it.s_right = it.s_right_next = -1;
        it.local = 0;
        it.K_inst = K[b];
        it.level = levels_for(K[b]);
        g.roots.push_back(it);
    }
}

}  // namespace fpsa
