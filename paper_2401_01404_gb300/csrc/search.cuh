// search.cuh -- scratch buffers of the best-pairs search (internal).
#pragma once

#include <vector>

#include "common.cuh"

struct SearchBufs {
    DBuf knn_id, knn_d, knn_new;                  // lists of the current level
    DBuf indeg, inoff, cursor, in_e;              // reverse edges
    DBuf in_last, in_fresh;                       // per list slot: iterations that took it into U
    DBuf U, Uf, Udeg, Usym;                       // undirected view
    DBuf scan_in, scan_tmp, scan_tmp2;            // scans
    DBuf cand, cand_d;                            // candidate pairs and scores
    DBuf seg_node, seg_start, seg_count, seg_vbase;  // candidates grouped by first node
    DBuf off_t, off_v, off_d, off_sv, off_sd;     // offers
    DBuf pairs_tmp;                               // scratch pair list
    DBuf ek, ev;                                  // edge sort
    DBuf dset;                                    // D membership set
    DBuf flag, pos;                               // compaction
    DBuf gid_a, gid_b;                            // level node sets
    DBuf ex_pairs, ex_d, ex_keys, ex_vals, dense;  // exhaustive scoring
    DBuf res_pairs, res_d;                        // collected pairs
    DBuf fk, fv, fk2, fv2;                        // final ordering
    DBuf out_pairs, out_d;                        // result
    DBuf sort_k2, sort_v2, sort_tmp;              // radix sort scratch
    DBuf scr_A, scr_B, scr_l1;                    // screen operands
    DBuf klen;                                    // per-node list lengths of the current level
    DBuf iter;                                    // device-side iteration counter
    DBuf g0_id, g0_d, g0_klen;                    // first-level lists, kept when a later level runs
    DBuf seed;                                    // device copy of the search's seed
    DBuf nnd_acc;                                 // the device loop's sums: candidates, dropped offers
    int64_t res_n = 0;
    int64_t klen_sum = 0;
    // the k-NN graph of the first level: rows g0_n, stride g0_K (0: no lists);
    // g0_moved: the lists were moved into g0_* when the second level started
    int64_t g0_n = 0;
    int g0_K = 0;
    bool g0_moved = false;

    std::vector<DBuf *> all() {
        return {&knn_id, &knn_d, &knn_new, &indeg, &inoff, &cursor, &in_e, &in_last, &in_fresh, &U, &Uf, &Udeg, &Usym,
                &scan_in, &scan_tmp, &scan_tmp2, &cand, &cand_d, &seg_node, &seg_start, &seg_count, &seg_vbase, &off_t, &off_v, &off_d, &off_sv,
                &off_sd, &pairs_tmp, &ek, &ev, &dset, &flag, &pos, &gid_a, &gid_b, &ex_pairs, &ex_d,
                &ex_keys, &ex_vals, &dense, &res_pairs, &res_d, &fk, &fv, &fk2, &fv2, &out_pairs,
                &out_d, &sort_k2, &sort_v2, &sort_tmp, &scr_A, &scr_B, &scr_l1, &klen, &iter, &g0_id, &g0_d, &g0_klen, &seed, &nnd_acc};
    }
};

void free_search_bufs(SearchBufs *sb);
recon_status score_pairs_device(recon_ctx *c, const int32_t *pairs, int64_t P, const int32_t *gid, float *d,
                                float *w);
recon_status findbest_run(recon_ctx *c, int k_cfg, int64_t m, int32_t **pairs_dev, float **d_dev, int64_t *count);
recon_status screen_run(recon_ctx *c, int64_t m, int32_t **pairs_dev, float **d_dev, int64_t *count);
recon_status exhaustive_run(recon_ctx *c, int64_t m, int32_t **pairs_dev, float **d_dev, int64_t *count);
recon_status select_run(recon_ctx *c, const int32_t *pairs, const float *d, int64_t P, int64_t m, int32_t **pairs_dev,
                        float **d_dev, int64_t *count);
recon_status row_best_run(recon_ctx *c, const int32_t *rows_dev, int64_t nrows, float cut, int32_t **pairs_dev,
                          float **d_dev, int64_t *count);
recon_status knn_graph_copy(recon_ctx *c, int32_t *ids, float *d, int64_t cap, int32_t *k_out, int64_t *n_out);
