// proposal.cuh -- state of the learned proposal (internal).
#pragma once

#include "common.cuh"

#define PROP_SKETCH 64
#define PROP_HIDDEN 128
#define PROP_EMBED 32

struct Proposal {
    DBuf w, m1, m2, g;        // FP32 parameters, Adam moments, gradient
    DBuf w1b, w2b;            // BF16 copies used by the forward pass
    DBuf omega, sketch;       // sketch matrix (bits) and node sketches
    DBuf emb, act, de, dA;    // embeddings, first-layer pre-activations, gradients
    DBuf tpairs, ttau, loss;  // training pairs, targets, loss accumulator
    DBuf seedA;               // bf16 embedding operands for seeding
    // seeding scratch, kept between searches
    DBuf s_pairs, s_vals, s_cands, s_ot, s_ov, s_od, s_cnt, s_offw, s_off, s_cur, s_sv, s_sd, s_tmp;
    bool ready = false;
    bool trained = false;     // set by recon_proposal_train; learned seeding needs it
    int64_t t = 0;            // Adam step
    uint64_t omega_seed = 0;
};

int64_t proposal_param_count();
cudaError_t proposal_setup(recon_ctx *c, Proposal &P, uint64_t seed);
cudaError_t proposal_forward(recon_ctx *c, Proposal &P, bool keep_act);
cudaError_t proposal_resketch(recon_ctx *c, Proposal &P, uint64_t seed);
cudaError_t proposal_grad(recon_ctx *c, Proposal &P, const int32_t *pairs, const float *tau, int64_t n,
                          double *loss_dev);
cudaError_t proposal_adam(recon_ctx *c, Proposal &P, float lr);
cudaError_t proposal_seed_operands(recon_ctx *c, Proposal &P, void *A);
void free_proposal(Proposal *P);
recon_status learned_seed_lists(recon_ctx *c, int n, int K, const int32_t *klen, uint64_t seed, int32_t *ids,
                                int64_t *nseeded_out);
