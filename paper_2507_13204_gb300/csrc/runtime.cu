// Host runtime of libkg.so: handles, validation, workspaces, error reporting,
// and dispatch to the per-kind kernels.  Every exported function returns a
// kg_status and never aborts.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kg_device.cuh"
#include "kg_internal.h"

namespace kg {

// One warp waits, through the same bounded wait as the TMA pipelines, on an
// mbarrier that nothing arrives at and no copy completes: the wait gives up
// after limit_ns, the kernel records ERRBIT_TIMEOUT and returns normally.
__global__ void bounded_wait_check_kernel(uint64_t limit_ns, unsigned* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
  if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) set_error(err, ERRBIT_TIMEOUT);
}

static thread_local std::string t_msg;
static thread_local int t_launches = 0;
static std::atomic<long> g_alloc_count{0};

kg_status fail(kg_status st, const std::string& msg) {
  t_msg = msg;
  return st;
}

kg_status cuda_fail(cudaError_t e, const char* what) {
  t_msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? KG_ERR_OOM : KG_ERR_CUDA;
}

void count_launch(int k) { t_launches += k; }

// ---- main-kernel timing -------------------------------------------------
namespace {
struct ProfState {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, stop), reused across enables
  int used = 0;                 // events recorded since enable
  const char* name = "";
};
thread_local ProfState t_prof;
constexpr int kMaxProfLaunches = 65536;
}  // namespace

void prof_begin(cudaStream_t s, const char* name) {
  ProfState& P = t_prof;
  if (!P.on || P.used / 2 >= kMaxProfLaunches) return;
  while ((int)P.ev.size() < P.used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    P.ev.push_back(e);
  }
  if (cudaEventRecord(P.ev[P.used], s) == cudaSuccess) {
    P.name = name;
    P.used += 1;
  }
}

void prof_end(cudaStream_t s) {
  ProfState& P = t_prof;
  if (!P.on || (P.used & 1) == 0) return;
  if (cudaEventRecord(P.ev[P.used], s) == cudaSuccess) P.used += 1;
  else P.used -= 1;
}
void reset_launch_count() { t_launches = 0; }

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  long n = ++g_alloc_count;
  if (const char* env = std::getenv("KG_TEST_FAIL_ALLOC")) {
    long target = std::atol(env);
    if (target > 0 && n == target) return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes < 16 ? 16 : bytes);
}

cudaError_t set_smem_once(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> bytes set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find({fn, dev});
  if (it != done.end() && it->second == bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[{fn, dev}] = bytes;
  return e;
}

int num_sms() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      sms = 152;
  });
  return sms;
}

kg_status ws_alloc(kg_problem* p, void** out, size_t bytes, const char* what) {
  void* ptr = nullptr;
  cudaError_t e = dev_alloc(&ptr, bytes);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(KG_ERR_OOM, std::string("workspace allocation failed (") + what + ", " +
                                std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
  }
  p->allocs.push_back(ptr);
  p->ws_bytes += bytes;
  *out = ptr;
  return KG_OK;
}

kg_status ws_common(kg_problem* p, int fpart_len, cudaStream_t s) {
  kg_status rc;
  if ((rc = ws_alloc(p, (void**)&p->err, 16, "error word")) != KG_OK) return rc;
  if ((rc = ws_alloc(p, (void**)&p->counter, 16, "arrival counter")) != KG_OK) return rc;
  if ((rc = ws_alloc(p, (void**)&p->fpart, sizeof(double) * (size_t)fpart_len, "f partials")) != KG_OK)
    return rc;
  p->fpart_len = fpart_len;
  cudaError_t e;
  if ((e = cudaMemsetAsync(p->err, 0, 16, s)) != cudaSuccess) return cuda_fail(e, "zero error word");
  if ((e = cudaMemsetAsync(p->counter, 0, 16, s)) != cudaSuccess) return cuda_fail(e, "zero counter");
  return KG_OK;
}

}  // namespace kg

using namespace kg;

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static void free_problem(kg_problem* p) {
  if (!p) return;
  for (void* a : p->allocs) cudaFree(a);
  delete p;
}

extern "C" {

void kg_options_default(kg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dtype = KG_F64;
  o->strategy = KG_STRATEGY_AUTO;
  o->mode = KG_MODE_AUTO;
  o->arith = KG_ARITH_AUTO;
}

const char* kg_last_error(void) { return t_msg.c_str(); }

static int env_choice(const char* name, const char* const* words, const int* values, int count,
                      int* out) {
  const char* v = std::getenv(name);
  if (!v || !*v) return 0;
  for (int i = 0; i < count; ++i)
    if (std::strcmp(v, words[i]) == 0) {
      *out = values[i];
      return 0;
    }
  std::string allowed;
  for (int i = 0; i < count; ++i) allowed += (i ? "|" : "") + std::string(words[i]);
  fail(KG_ERR_INVALID_ARG, std::string(name) + "=" + v + ": expected one of " + allowed);
  return -1;
}

kg_status kg_options_apply_env(kg_options* o) {
  if (!o) return fail(KG_ERR_INVALID_ARG, "kg_options_apply_env: NULL options");
  static const char* const sw[] = {"auto", "atomic", "csr", "transpose", "fused", "shared", "warp",
                                   "tile"};
  static const int sv[] = {KG_STRATEGY_AUTO, KG_STRATEGY_ATOMIC, KG_STRATEGY_CSR,
                           KG_STRATEGY_TRANSPOSE, KG_STRATEGY_FUSED, KG_STRATEGY_SHARED,
                           KG_STRATEGY_WARP, KG_STRATEGY_TILE};
  static const char* const mw[] = {"auto", "recompute", "tape"};
  static const int mv[] = {KG_MODE_AUTO, KG_MODE_RECOMPUTE, KG_MODE_TAPE};
  static const char* const aw[] = {"auto", "native", "pair"};
  static const int av[] = {KG_ARITH_AUTO, KG_ARITH_NATIVE, KG_ARITH_PAIR};
  static const char* const cw[] = {"0", "1"};
  static const int cv[] = {0, 1};
  kg_options r = *o;
  if (env_choice("KG_STRATEGY", sw, sv, 8, &r.strategy) || env_choice("KG_MODE", mw, mv, 3, &r.mode) ||
      env_choice("KG_ARITH", aw, av, 3, &r.arith) || env_choice("KG_CHECK", cw, cv, 2, &r.check))
    return KG_ERR_INVALID_ARG;
  *o = r;
  return KG_OK;
}

kg_status kg_tape_generation(const kg_problem* p, uint64_t* gen) {
  if (!p || !gen) return fail(KG_ERR_INVALID_ARG, "kg_tape_generation: NULL argument");
  *gen = p->tape_gen;
  return KG_OK;
}

int kg_last_launch_count(void) { return t_launches; }

kg_status kg_profile_enable(int on) {
  t_prof.on = on != 0;
  t_prof.used = 0;
  return KG_OK;
}

kg_status kg_profile_read(double* ms, int* launches, const char** name) {
  ProfState& P = t_prof;
  double tot = 0.0;
  int pairs = P.used / 2;
  for (int i = 0; i < pairs; ++i) {
    cudaError_t e = cudaEventSynchronize(P.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "kg_profile_read");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, P.ev[2 * i], P.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "kg_profile_read");
    tot += t;
  }
  if (ms) *ms = tot;
  if (launches) *launches = pairs;
  if (name) *name = P.name;
  return KG_OK;
}

size_t kg_workspace_bytes(const kg_problem* p) { return p ? p->ws_bytes : 0; }

kg_status kg_get_config(const kg_problem* p, int* strategy, int* mode, int* arith) {
  if (!p) return fail(KG_ERR_INVALID_ARG, "kg_get_config: NULL problem");
  if (strategy) *strategy = p->strategy;
  if (mode) *mode = p->mode;
  if (arith) *arith = p->arith;
  return KG_OK;
}

kg_status kg_create(kg_problem** out, int kind, const int64_t* sizes, int nsizes,
                    const void* const* data, int ndata, const kg_options* opt, kg_stream s) {
  t_msg.clear();
  if (!out) return fail(KG_ERR_INVALID_ARG, "kg_create: out is NULL");
  *out = nullptr;
  if (!sizes || nsizes < 1) return fail(KG_ERR_INVALID_ARG, "kg_create: sizes missing");
  for (int i = 0; i < nsizes; ++i) {
    const int64_t lo = (kind == KG_SPQUADFORM && i == 2) ? 0 : 1;  // nnz may be 0
    if (sizes[i] < lo || sizes[i] >= (int64_t(1) << 31))
      return fail(KG_ERR_INVALID_ARG, "kg_create: every size must be in [1, 2^31) (nnz in [0, 2^31))");
  }
  kg_options o;
  kg_options_default(&o);
  if (opt) o = *opt;
  if (kg_options_apply_env(&o) != KG_OK) return KG_ERR_INVALID_ARG;
  if (o.dtype != KG_F64 && o.dtype != KG_F32)
    return fail(KG_ERR_INVALID_ARG, "kg_create: dtype must be KG_F64 or KG_F32");
  if (o.strategy < KG_STRATEGY_AUTO || o.strategy > KG_STRATEGY_TILE)
    return fail(KG_ERR_INVALID_ARG, "kg_create: bad strategy");
  if (o.mode < KG_MODE_AUTO || o.mode > KG_MODE_TAPE)
    return fail(KG_ERR_INVALID_ARG, "kg_create: bad mode");
  if (o.arith < KG_ARITH_AUTO || o.arith > KG_ARITH_PAIR)
    return fail(KG_ERR_INVALID_ARG, "kg_create: bad arith");
  if (o.block < 0 || o.block > 1024 || (o.block % 32) != 0)
    return fail(KG_ERR_INVALID_ARG, "kg_create: block must be 0 or a multiple of 32 <= 1024");
  if (o.team < 0 || o.tile < 0) return fail(KG_ERR_INVALID_ARG, "kg_create: team/tile < 0");

  kg_problem* p = new (std::nothrow) kg_problem();
  if (!p) return fail(KG_ERR_OOM, "kg_create: host allocation failed");
  p->kind = kind;
  p->dtype = o.dtype;
  p->opt = o;
  p->esize = o.dtype == KG_F64 ? 8 : 4;
  p->strategy = o.strategy;
  p->mode = o.mode;
  p->arith = o.arith;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  p->last_stream = st;

  kg_status rc = KG_OK;
  switch (kind) {
    case KG_QUADFORM:
      if (nsizes > 2 || !data || ndata < 1 || !data[0]) {
        rc = fail(KG_ERR_INVALID_ARG, "kg_create(QUADFORM): sizes {n} or {m,n}; data {A}");
        break;
      }
      p->m = sizes[0];
      p->n = nsizes == 2 ? sizes[1] : sizes[0];
      if (p->m * p->n >= (int64_t(1) << 40)) {
        rc = fail(KG_ERR_INVALID_ARG, "kg_create(QUADFORM): m*n too large");
        break;
      }
      p->data0 = data[0];
      if (!aligned16(p->data0)) {
        rc = fail(KG_ERR_INVALID_ARG, "kg_create(QUADFORM): A must be 16-byte aligned");
        break;
      }
      rc = qf_setup(p, st);
      break;
    case KG_TETENERGY:
      if (nsizes != 2 || !data || ndata < 2 || !data[0] || !data[1]) {
        rc = fail(KG_ERR_INVALID_ARG, "kg_create(TETENERGY): sizes {N_e, N_v}; data {conn, G}");
        break;
      }
      p->m = sizes[0];
      p->n = sizes[1];
      p->data0 = data[0];
      p->data1 = data[1];
      if (!aligned16(p->data0) || !aligned16(p->data1)) {
        rc = fail(KG_ERR_INVALID_ARG, "kg_create(TETENERGY): conn and G must be 16-byte aligned");
        break;
      }
      rc = tet_setup(p, st);
      break;
    case KG_SPQUADFORM:
      if (nsizes != 3 || !data || ndata < 3 || !data[0] || (sizes[2] > 0 && (!data[1] || !data[2]))) {
        rc = fail(KG_ERR_INVALID_ARG, "kg_create(SPQUADFORM): sizes {m, n, nnz}; data {rowptr, col, val}");
        break;
      }
      p->m = sizes[0];
      p->n = sizes[1];
      p->nnz = sizes[2];
      p->data0 = data[0];
      p->data1 = data[1];
      p->data2 = data[2];
      rc = spq_setup(p, st);
      break;
    case KG_LAPLACE1D:
      if (nsizes != 1 || !data || ndata < 1 || !data[0]) {
        rc = fail(KG_ERR_INVALID_ARG, "kg_create(LAPLACE1D): sizes {n}; data {b}");
        break;
      }
      p->n = p->m = sizes[0];
      p->data0 = data[0];
      rc = lap_setup(p, st);
      break;
    default:
      rc = fail(KG_ERR_INVALID_ARG, "kg_create: unknown kind " + std::to_string(kind));
  }
  if (rc == KG_OK) {
    // host staging for kg_grad_host, and the error word
    size_t vec = (size_t)(p->kind == KG_TETENERGY ? p->n : p->n) * p->esize;
    if ((rc = ws_alloc(p, &p->xdev, vec, "host-call x")) == KG_OK &&
        (rc = ws_alloc(p, &p->gdev, vec, "host-call gx")) == KG_OK &&
        (rc = ws_alloc(p, &p->fdev, 16, "host-call f")) == KG_OK) {
    }
  }
  if (rc == KG_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "kg_create: set-up kernels");
  }
  if (rc == KG_OK && p->err) {
    unsigned h = 0;
    cudaError_t e = cudaMemcpy(&h, p->err, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "kg_create: reading error word");
    else if (h & ERRBIT_BOUNDS)
      rc = fail(KG_ERR_BOUNDS, p->kind == KG_SPQUADFORM
                                   ? "kg_create: CSR structure invalid (rowptr or a column out of range)"
                                   : "kg_create: connectivity entry outside [0, N_v)");
  }
  if (rc != KG_OK) {
    std::string keep = t_msg;
    free_problem(p);
    t_msg = keep;
    return rc;
  }
  *out = p;
  return KG_OK;
}

kg_status kg_eval(kg_problem* p, const void* x, void* f, kg_stream s) {
  reset_launch_count();
  if (!p || !x || !f) return fail(KG_ERR_INVALID_ARG, "kg_eval: NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  p->last_stream = st;
  switch (p->kind) {
    case KG_QUADFORM: return qf_eval(p, x, f, st);
    case KG_TETENERGY: return tet_eval(p, x, f, false, st);
    case KG_LAPLACE1D: return lap_eval(p, x, f, st);
    case KG_SPQUADFORM: return spq_eval(p, x, f, st);
  }
  return fail(KG_ERR_STATE, "kg_eval: corrupt handle");
}

kg_status kg_grad(kg_problem* p, const void* x, void* f, void* gx, void* gdata, const void* seed,
                  int accumulate, kg_stream s) {
  reset_launch_count();
  if (!p || !x || !gx) return fail(KG_ERR_INVALID_ARG, "kg_grad: NULL argument");
  if (accumulate != 0 && accumulate != 1)
    return fail(KG_ERR_INVALID_ARG, "kg_grad: accumulate must be 0 or 1");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  p->last_stream = st;
  switch (p->kind) {
    case KG_QUADFORM: return qf_grad(p, x, f, gx, gdata, seed, accumulate, st);
    case KG_TETENERGY:
      if (gdata) return fail(KG_ERR_UNSUPPORTED, "kg_grad(TETENERGY): no gradient w.r.t. G");
      return tet_grad(p, x, f, gx, seed, accumulate, st);
    case KG_LAPLACE1D: return lap_grad(p, x, f, gx, gdata, seed, accumulate, st);
    case KG_SPQUADFORM: return spq_grad(p, x, f, gx, gdata, seed, accumulate, st);
  }
  return fail(KG_ERR_STATE, "kg_grad: corrupt handle");
}

kg_status kg_eval_tape(kg_problem* p, const void* x, void* f, kg_stream s) {
  reset_launch_count();
  if (!p || !x) return fail(KG_ERR_INVALID_ARG, "kg_eval_tape: NULL argument");
  if (p->kind != KG_TETENERGY && p->kind != KG_LAPLACE1D)
    return fail(KG_ERR_UNSUPPORTED, "kg_eval_tape: TETENERGY and LAPLACE1D only");
  if (!p->tape) return fail(KG_ERR_STATE, "kg_eval_tape: problem was not created in TAPE mode");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  p->last_stream = st;
  if (p->kind == KG_LAPLACE1D) return lap_eval_tape(p, x, f, st);
  return tet_eval(p, x, f, true, st);
}

kg_status kg_hvp(kg_problem* p, const void* x, const void* v, void* hv, const void* seed,
                 int accumulate, kg_stream s) {
  reset_launch_count();
  if (!p || !v || !hv) return fail(KG_ERR_INVALID_ARG, "kg_hvp: NULL argument");
  if (accumulate != 0 && accumulate != 1)
    return fail(KG_ERR_INVALID_ARG, "kg_hvp: accumulate must be 0 or 1");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  p->last_stream = st;
  switch (p->kind) {
    // ||A x||^2 is a homogeneous quadratic: its Hessian times v is its gradient at v
    case KG_QUADFORM: return qf_grad(p, v, p->fdev, hv, nullptr, seed, accumulate, st);
    case KG_SPQUADFORM: return spq_grad(p, v, p->fdev, hv, nullptr, seed, accumulate, st);
    case KG_LAPLACE1D: return lap_hvp(p, v, hv, seed, accumulate, st);
    case KG_TETENERGY:
      if (!x) return fail(KG_ERR_INVALID_ARG, "kg_hvp: x is NULL");
      return tet_hvp(p, x, v, hv, seed, accumulate, st);
  }
  return fail(KG_ERR_INVALID_ARG, "kg_hvp: bad problem");
}

kg_status kg_grad_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate,
                            kg_stream s) {
  reset_launch_count();
  if (!p || !gx) return fail(KG_ERR_INVALID_ARG, "kg_grad_from_tape: NULL argument");
  if (p->kind != KG_TETENERGY && p->kind != KG_LAPLACE1D)
    return fail(KG_ERR_UNSUPPORTED, "kg_grad_from_tape: TETENERGY and LAPLACE1D only");
  if (!p->tape || !p->tape_valid)
    return fail(KG_ERR_STATE, "kg_grad_from_tape: no tape recorded (call kg_eval_tape first)");
  if (accumulate != 0 && accumulate != 1)
    return fail(KG_ERR_INVALID_ARG, "kg_grad_from_tape: accumulate must be 0 or 1");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  p->last_stream = st;
  if (p->kind == KG_LAPLACE1D) return lap_grad_from_tape(p, gx, seed, accumulate, st);
  return tet_grad_from_tape(p, gx, seed, accumulate, st);
}

kg_status kg_grad_host(kg_problem* p, const void* x_host, void* f_host, void* gx_host,
                       kg_stream s) {
  if (!p || !x_host || !gx_host) return fail(KG_ERR_INVALID_ARG, "kg_grad_host: NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  size_t bytes = (size_t)p->n * p->esize;
  cudaError_t e = cudaMemcpyAsync(p->xdev, x_host, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "kg_grad_host: copy x");
  kg_status rc = kg_grad(p, p->xdev, p->fdev, p->gdev, nullptr, nullptr, 0, s);
  if (rc != KG_OK) return rc;
  e = cudaMemcpyAsync(gx_host, p->gdev, bytes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "kg_grad_host: copy gx");
  if (f_host) {
    e = cudaMemcpyAsync(f_host, p->fdev, p->esize, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "kg_grad_host: copy f");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "kg_grad_host: synchronize");
  return KG_OK;
}

kg_status kg_sync(kg_problem* p) {
  if (!p) return fail(KG_ERR_INVALID_ARG, "kg_sync: NULL problem");
  cudaError_t e = cudaStreamSynchronize(p->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "kg_sync: synchronize");
  if (!p->err) return KG_OK;
  unsigned h = 0;
  e = cudaMemcpy(&h, p->err, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "kg_sync: read error word");
  if (h) {
    e = cudaMemset(p->err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "kg_sync: clear error word");
  }
  if (h & ERRBIT_BOUNDS) return fail(KG_ERR_BOUNDS, "device: connectivity entry outside [0, N_v)");
  if (h & ERRBIT_TIMEOUT) return fail(KG_ERR_TIMEOUT, "device: a bounded wait gave up");
  if (h & ERRBIT_RANGE)
    return fail(KG_ERR_RANGE, "device: an input is outside the float-pair range (0 or 2^-60 <= |v| < 2^40)");
  return KG_OK;
}

kg_status kg_check_bounded_wait(kg_problem* p, uint64_t limit_ns, kg_stream s) {
  reset_launch_count();
  if (!p || !p->err) return fail(KG_ERR_INVALID_ARG, "kg_check_bounded_wait: NULL problem");
  if (limit_ns == 0 || limit_ns > 2000000000ull)
    return fail(KG_ERR_INVALID_ARG, "kg_check_bounded_wait: limit_ns must be in (0, 2e9]");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  p->last_stream = st;
  bounded_wait_check_kernel<<<1, 32, 0, st>>>(limit_ns, p->err);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kg_check_bounded_wait");
  return KG_OK;
}

void kg_destroy(kg_problem* p) {
  if (!p) return;
  cudaStreamSynchronize(p->last_stream);
  free_problem(p);
}

}  // extern "C"
