// Launch descriptors of the search kernels (k_search.cu, k_scan_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "erq_internal.cuh"

namespace erq {

// Inputs/outputs of the planning kernels (probe lists -> work items).
struct PlanArgs {
    const int32_t* probe;       // [nq][probe_stride]
    int64_t probe_stride;
    const int32_t* npr_in;      // optional [nq]
    int npr_uniform;
    int64_t nq;
    int maxp, nlist, QT, RR;
    int two_phase = 0;          // nearest probed cluster of every query in a first phase of work items
    const int64_t* list_off;
    const int32_t* corder;      // [nlist] clusters by decreasing size
    int32_t* npr;               // [nq] effective nprobe
    int32_t* probe_c;           // [nq][maxp] validated cluster or -1
    int32_t* cnt_c;             // [2 nlist] queries per phase cluster (v = c: nearest probe, nlist + c: others)
    int32_t* pos_c;             // [2 nlist]
    int32_t* touch_c;           // [nlist] probes per cluster (distinct probed rows)
    int32_t* slot_nr;           // [nq][maxp] ranges of the slot's cluster
    int32_t* slot_off;          // [nq][maxp]
    int64_t* qtot;              // [nq]
    int64_t* qbase;             // [nq+1]
    int64_t* cnt64;             // [2 nlist]
    int64_t* items_c;           // [2 nlist]
    int64_t* qoff;              // [2 nlist + 1]
    int64_t* item_off;          // [2 nlist + 1]
    int64_t* qlist;             // [nq*maxp]
    uint32_t* status;
    const float* sqd;           // optional [nq][nlist] probe values (||q_r - c||^2, or -<q_r, c>): when given,
    float* dqc;                 //   the plan copies the probed pairs' values into dqc [nq][maxp]
    DevChecks ck;
    unsigned long long* stats;  // [4]: (query, candidate) pairs, rows of distinct probed clusters,
                                //      tensor-core row blocks, row blocks x padded queries (item tables)
};

struct ScanLaunch {
    const float* Qrot;
    const void* Qh;             // FP16 rotated queries (tensor-core path)
    const void* Q8;             // e4m3 rotated queries, rows of Dq bytes (kind::f8f6f4 path)
    const float* qscale;        // their per-query power-of-two scales
    int64_t Dq;
    uint32_t* status;
    int64_t N;
    const uint8_t* codes;
    const float* g_const;
    const float* f_res;
    const int64_t* list_off;
    const int64_t* list_ids;
    const int64_t* qlist;
    const int64_t* qoff;
    const int4* items;
    const int64_t* n_items;
    const float* dqc;
    const int32_t* slot_off;
    const int64_t* qbase;
    uint64_t* inter;
    int32_t* inter_cnt;
    const int4* itemd;          // tensor-core path: per-item {rb0 lo, rb0 hi, rows, queries}
    const int4* itemq;          // tensor-core path: per-item query slots
    const float4* rowmeta;      // tensor-core path: per padded row {g, f_res/2, id, 0}
    const uint64_t* codes_p;    // tensor-core path: packed B-bit codes, tiled and padded
    int64_t Np;                 // tensor-core path: padded rows
    unsigned long long* tq;     // tensor-core path: [nq] query-wide thresholds (all ones at the start)
    int maxp, D, B, kp, RR, nlist;
    int qn;                     // tensor-core path: queries per work item (32, 64 or 128)
    int64_t nq;                 // tensor-core path: query rows (extent of the gathered query matrix)
    unsigned int* work_ctr;     // tensor-core path: dynamic work-item counter, zero at launch
    unsigned long long wait_ns; // tensor-core path: limit of every bounded device-side wait (0 = default)
    long long stall_stage = -1; // tensor-core path: test stall of the bounded-wait path (-1 = none)
    int grid;
    int ip;                     // inner-product metric (per-row factor f_res / 4, no g; dqc holds -<c, q_r>)
    DevChecks ck;
};

// Two-stage (MSB-first) search, k_two_stage.cu.
struct TwoStageLaunch {
    const int32_t* probe_c;     // [nq][maxp] validated probes (-1: none)
    const float* dqc;           // [nq][maxp] ||q_r - c||^2
    const int64_t* list_off;
    const int64_t* poff;
    const uint64_t* codes_p;
    const float4* rowmeta;      // [Np] {g, f_res / 2, id, 0}
    const float4* meta1;        // [Np] {g1, f1 / 2, err1, 0} (stage-1 factors)
    const float* Qrot;          // [nq][D]
    float* T;                   // [nq][D / 4][16] workspace: plane-word nibble tables
    const int32_t* rbase;       // [nq][maxp] first row of each probe within its query
    const int64_t* qoffr;       // [nq + 1] first row slot of each query
    float* ub;                  // [rows] workspace
    float* lb;                  // [rows] workspace
    float* s1;                  // [rows] workspace
    float* tau;                 // [nq] out: pruning thresholds
    int32_t* scnt;              // [nq] out: survivors
    uint64_t* skey;             // [rows] workspace (also the threshold selection's scratch)
    uint32_t* scratch;          // [rows] u32 scratch (may alias skey)
    uint64_t* cand;             // [nq][kp] out: the k' best survivors' keys, ascending
    int64_t nq;
    int maxp, D, B, kp;
    float eps0;
};
cudaError_t launch_stage1_factors(const float* R, int64_t r0, int64_t m, int D, int B, const uint8_t* codes,
                                  const float* f_add, const float* Cp, const int32_t* cl_of_row,
                                  const int64_t* list_off, const int64_t* poff, float4* meta1, cudaStream_t s);
cudaError_t launch_two_stage_rows(const int32_t* probe_c, int64_t nq, int maxp, const int64_t* list_off,
                                  int32_t* rbase, int64_t* qrows, cudaStream_t s);
cudaError_t launch_two_stage(const TwoStageLaunch& L, cudaStream_t s);
cudaError_t launch_excl_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

cudaError_t launch_dqc(const float* Q, const float* C, const int32_t* probe, const int32_t* npr, int64_t nq, int maxp,
                       int D, int ip, float* dqc, cudaStream_t s);
cudaError_t launch_plan(const PlanArgs& p, cudaStream_t s);
cudaError_t launch_plan_items(const PlanArgs& p, int4* items, cudaStream_t s);
cudaError_t launch_scan_fp32(const ScanLaunch& L, cudaStream_t s);
size_t scan_fp32_smem(int kp);
int scan_fp32_blocks_per_sm(int kp, int B);   // resident FP32-scan blocks per SM at this k' and code width
int merge_sortn(int kp, int lstride);
cudaError_t launch_make_keys(const int64_t* ids, const float* vals, int64_t n, int64_t id_limit, int neg,
                             uint64_t* keys, cudaStream_t s);
cudaError_t launch_keys_to_pairs(const uint64_t* keys, int64_t n, int neg, int64_t* ids, float* vals, cudaStream_t s);
cudaError_t launch_one_list_per_query(int64_t nq, int m, int32_t* counts, int64_t* off, cudaStream_t s);
cudaError_t launch_merge(const uint64_t* inter, const int32_t* inter_cnt, const int64_t* qbase, int64_t nq, int kp,
                         int lstride, uint64_t* cand, const DevChecks& ck, cudaStream_t s);
int scan_list_stride(int precision, int kp, int qn);
cudaError_t launch_item_tables(const int4* items, const int64_t* n_items, int64_t items_bound, const int64_t* list_off,
                               const int64_t* poff, const int64_t* qoff, const int64_t* qlist, const float* dqc,
                               const int64_t* qbase, const int32_t* slot_off, int maxp, int RR, int qn, int nlist,
                               int4* itemd,
                               int4* itemq, unsigned long long* stats, const DevChecks& ck, cudaStream_t s);
bool scan_tc_shape_ok(int qn, int kp);
cudaError_t launch_scan_layout(const uint8_t* codes, const float* g, const float* f_res, const int64_t* ids,
                               const int64_t* list_off, const int64_t* poff, int nlist, int64_t Np, int D, int B,
                               uint64_t* codes_p, float4* rowmeta, cudaStream_t s);
cudaError_t launch_quant_e4m3(const float* x, int64_t n, int D, int Dq, int dup, unsigned char* y, float* scale,
                              cudaStream_t s);
cudaError_t launch_rerank(const uint64_t* cand, int64_t nq, int kp, const float* X, const float* Q, int D, int k,
                          int do_rerank, int ip, int64_t* ids, float* dists, int64_t* cand_ids, float* cand_est,
                          const DevChecks& ck, cudaStream_t s);
cudaError_t launch_estimate(const float* Q, const float* Qrot, const int64_t* ids, int64_t nq, int nc,
                            const erq_index* ix, int ipm, float* est, cudaStream_t s);
cudaError_t launch_backward_gather(const float* Q, const int64_t* ids, const float* gs, int64_t nq, int nc,
                                   const erq_index* ix, int ipm, float* V, float* Wv, cudaStream_t s);

}  // namespace erq
