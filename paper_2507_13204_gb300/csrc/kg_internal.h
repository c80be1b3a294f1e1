// Internal declarations shared by the translation units of libkg.so.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/kg.h"
#include "kg_pair.cuh"

namespace kg {

// Bits of the sticky device error word.
enum : unsigned { ERRBIT_BOUNDS = 1u, ERRBIT_TIMEOUT = 2u, ERRBIT_RANGE = 4u };

// Status + thread-local message.
kg_status fail(kg_status st, const std::string& msg);
kg_status cuda_fail(cudaError_t e, const char* what);
void count_launch(int k = 1);
// Main-kernel timing (kg_profile_enable): brackets one launch with events.
void prof_begin(cudaStream_t s, const char* name);
void prof_end(cudaStream_t s);
void reset_launch_count();

// Allocation through one hook so that tests can force an allocation failure
// (environment variable KG_TEST_FAIL_ALLOC=N fails the N-th allocation).
cudaError_t dev_alloc(void** p, size_t bytes);

int num_sms();

// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes), made once per
// kernel, device and size: the per-call launch paths go through this.
cudaError_t set_smem_once(const void* fn, int bytes);
template <typename K>
inline cudaError_t set_smem_once(K* fn, size_t bytes) {
  return set_smem_once(reinterpret_cast<const void*>(fn), (int)bytes);
}

// Launch configuration of one dense row-team kernel.
struct QfConfig {
  int block = 256;  // threads per CTA
  int team = 256;   // threads per row team (32..block, power of 2)
  int cpt = 1;      // columns per team thread (compile-time variant)
  int grid = 1;     // CTAs
  int rows_per_cta = 1;
  int streamed = 0;  // 1: FP32 TMA-streamed kernel (quadform_f32.cu)
  int coop = 0;      // 1: the streamed gradient (pair, FP32) reduces its partials in one cooperative launch
};

struct kg_problem_impl;
}  // namespace kg

// Problem handle.  All device workspaces are owned here and allocated in
// kg_create; per-call entry points only launch kernels.
struct kg_problem {
  int kind = 0;
  int dtype = KG_F64;
  kg_options opt{};
  int strategy = KG_STRATEGY_AUTO;  // resolved strategy
  int mode = KG_MODE_RECOMPUTE;     // resolved mode
  int arith = KG_ARITH_NATIVE;      // resolved FP64 arithmetic
  int64_t m = 0, n = 0;             // QUADFORM m x n; TET m = N_e, n = N_v; LAPLACE1D n;
                                    // SPQUADFORM m x n
  int64_t nnz = 0;                  // SPQUADFORM stored entries
  const void* data0 = nullptr;      // A | conn | b | rowptr
  const void* data1 = nullptr;      // - | G | - | col
  const void* data2 = nullptr;      // - | - | - | val
  size_t esize = 8;

  // workspaces
  std::vector<void*> allocs;
  size_t ws_bytes = 0;
  void* partials = nullptr;  // dense: [grid][n] of T (FUSED / TRANSPOSE)
  double* fpart = nullptr;   // per-CTA f partials
  int fpart_len = 0;
  unsigned* counter = nullptr;
  unsigned* err = nullptr;   // sticky error word
  void* y = nullptr;         // dense / 1-D: forward intermediates
  void* tape = nullptr;      // tet: c_e [N_e][4]
  void* aprep = nullptr;     // FP64 pair: A (dense) or G (tet) split into float pairs
  bool tape_valid = false;
  uint64_t tape_gen = 0;     // launches that wrote the tape (kg_tape_generation)
  int* rowptr = nullptr;     // tet CSR: [N_v + 2]; sparse CSC: colptr [n + 1]
  int* inc = nullptr;        // tet CSR: slots (tile * 128 + j) by vertex; sparse CSC: row of each entry
  void* valT = nullptr;      // sparse CSC: values in column order
  void* usplit = nullptr;    // tet pair: u and v as float pairs [2][N_v], split per call
  // tet TILE strategy (tet_tile.cu): per tile of 32 elements, its distinct
  // vertices and their incidence lists, built at kg_create
  int* tile_nv = nullptr;
  int* tile_vlist = nullptr;
  uint8_t* tile_vptr = nullptr;
  uint8_t* tile_inc = nullptr;
  int ntiles = 0;
  void* tile_part = nullptr;  // tet CSR strategy: the tile vertex sums [tile][128]
  void* xdev = nullptr;      // kg_grad_host staging
  void* gdev = nullptr;
  void* fdev = nullptr;

  kg::QfConfig qf;           // dense launch configuration
  int tet_block = 256, tet_grid = 1;
  int sq_team = 8, sq_col_team = 8;  // sparse: lanes per row team / per column team
  cudaStream_t last_stream = nullptr;
};

namespace kg {
// Per-kind entry points (defined in quadform.cu, tet.cu, laplace1d.cu).
kg_status qf_setup(kg_problem* p, cudaStream_t s);
kg_status qf_eval(kg_problem* p, const void* x, void* f, cudaStream_t s);
kg_status qf_grad(kg_problem* p, const void* x, void* f, void* gx, void* gA, const void* seed,
                  int accumulate, cudaStream_t s);

kg_status qf_native_fused_on_scratch(const double* A, int64_t m, int64_t n, const double* x,
                                     double* f, double* gx, double* scratch,
                                     size_t scratch_doubles, cudaStream_t s);

// FP32 TMA-streamed dense kernels (quadform_f32.cu)
bool qf_f32_supported(const kg_problem* p);
int qf_f32_grid(const kg_problem* p, int* band);
kg_status qf_f32_eval(kg_problem* p, const void* x, void* f, cudaStream_t s);
kg_status qf_f32_grad(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                      int accumulate, cudaStream_t s);

// float-pair dense kernels (quadform_pair.cu)
bool qf_pair_supported(const kg_problem* p);
kg_status pair_range_ok(kg_problem* p, const double* data, int64_t count, cudaStream_t s, bool* ok);
kg_status qf_pair_range_ok(kg_problem* p, cudaStream_t s, bool* ok);
kg_status qf_pair_prepare(kg_problem* p, cudaStream_t s);
// dst[i] = float pair (h, l) of src[i] for i < count (src and dst 16-byte aligned)
kg_status pair_prepare(const double* src, void* dst, int64_t count, cudaStream_t s);
int qf_pair_grid(const kg_problem* p, int* band);
// Whether the warp-specialized pair gradient can run as one cooperative launch
// (its whole grid resident at once); the test hook KG_TEST_NO_COOP=1 says no.
bool qf_pair_coop_fits(const kg_problem* p);
// The same for the FP32 streamed gradient (quadform_f32.cu).
bool qf_f32_coop_fits(const kg_problem* p);
kg_status qf_pair_eval(kg_problem* p, const void* x, void* f, cudaStream_t s);
kg_status qf_pair_grad(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                       int accumulate, cudaStream_t s);

// log1p table (256 float4 per device, uploaded once) and constants (tet_pair.cu)
kg_status logtab_for_device(const float4** out);
LogConsts log_consts();

// staged tet kernels (tet_pair.cu); mode 0 eval, 1 grad, 2 tape, 3 Hessian-vector
// product in direction v
int tet_staged_grid(const kg_problem* p);
kg_status tet_staged_setup(kg_problem* p);
// zero_gx: gx is zeroed by the pair kernels' vertex-split launch (pair GRAD / HVP only)
kg_status tet_staged(kg_problem* p, int mode, const void* x, void* f, void* gx, const void* seed,
                     cudaStream_t s, const void* v = nullptr, bool zero_gx = false);

kg_status tet_setup(kg_problem* p, cudaStream_t s);
kg_status tet_eval(kg_problem* p, const void* x, void* f, bool tape, cudaStream_t s);
kg_status tet_grad(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                   int accumulate, cudaStream_t s);
kg_status tet_grad_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate,
                             cudaStream_t s);
kg_status tet_hvp(kg_problem* p, const void* x, const void* v, void* hv, const void* seed,
                  int accumulate, cudaStream_t s);

// tiled reverse pass (tet_tile.cu): whether it applies, its create-time build,
// and one value-and-gradient (mode TS_GRAD) or Hessian-vector product (TS_HVP)
// from the float pairs of u (and v) split this call
bool tet_tile_supported(const kg_problem* p);
kg_status tet_tile_setup(kg_problem* p, cudaStream_t s);
kg_status tet_tile_run(kg_problem* p, int mode, const float2* us, const float2* vs, void* f, void* gx,
                       const void* seed, cudaStream_t s);
kg_status tet_tile_run_f32(kg_problem* p, int mode, const void* x, const void* v, void* f, void* gx,
                           const void* seed, cudaStream_t s);
// reproducible CSR strategy on the tiles: set-up (tiles, partials, vertex ->
// slot buckets; synchronises s) and the vertex gather of the tile partials
kg_status tet_tile_csr_setup(kg_problem* p, cudaStream_t s);
kg_status tet_tile_gather(kg_problem* p, void* gx, int accumulate, cudaStream_t s);
// reverse pass from the tape over the tiles (CSR: partials then gather; TILE:
// one reduction per tile vertex)
kg_status tet_tile_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate, cudaStream_t s);
// u (and v) of a float-pair tet problem split into float pairs in the
// problem's workspace, gx zeroed when zero_gx (tet_pair.cu); *us / *vs receive
// the pairs
kg_status tet_split_vertex_values(kg_problem* p, const void* x, const void* v, void* gx, bool zero_gx,
                                  const float2** us, const float2** vs, cudaStream_t s);

// In-place exclusive scan of data[0..n) into data[0..n] (data[n] = total; one
// CTA, set-up only; tet.cu).
void scan_exclusive(int* data, int n, cudaStream_t s);

// Buckets of positions by key (transposed index lists; tet.cu), synchronises s.
kg_status build_buckets(const int* keys, int64_t count, int nbins, int* binptr, int* perm,
                        cudaStream_t s);

// sparse ||A x||^2 (spquadform.cu)
kg_status spq_setup(kg_problem* p, cudaStream_t s);
kg_status spq_eval(kg_problem* p, const void* x, void* f, cudaStream_t s);
kg_status spq_grad(kg_problem* p, const void* x, void* f, void* gx, void* gval, const void* seed,
                   int accumulate, cudaStream_t s);

kg_status lap_setup(kg_problem* p, cudaStream_t s);
kg_status lap_eval(kg_problem* p, const void* x, void* f, cudaStream_t s);
kg_status lap_grad(kg_problem* p, const void* x, void* f, void* gx, void* gb, const void* seed,
                   int accumulate, cudaStream_t s);
kg_status lap_eval_tape(kg_problem* p, const void* x, void* f, cudaStream_t s);
kg_status lap_hvp(kg_problem* p, const void* v, void* hv, const void* seed, int accumulate,
                  cudaStream_t s);
kg_status lap_grad_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate,
                             cudaStream_t s);

// Workspace helper: allocate, record for kg_destroy, count bytes.
kg_status ws_alloc(kg_problem* p, void** out, size_t bytes, const char* what);
// Error word, arrival counter and `fpart_len` per-CTA f partials, zeroed on `s`.
kg_status ws_common(kg_problem* p, int fpart_len, cudaStream_t s);
}  // namespace kg
