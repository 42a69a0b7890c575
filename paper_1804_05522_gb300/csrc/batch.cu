// Batches of independent implicit-Euler instances (1D and 2D, uneven N, α and
// coefficients): host worker threads, each with its own CUDA stream, advance
// disjoint subsets of the instances so that small and large problems overlap
// on the GPU.  The HODLR leaf size of each (dimension, N) bucket can be chosen
// by timing trial steps of its first instance; choices are cached per process.
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <utility>
#include <vector>

#include "hodlr_internal.cuh"

namespace {

struct LeafKey {
  int dim, N, prec;
  bool operator<(const LeafKey& o) const {
    return std::tie(dim, N, prec) < std::tie(o.dim, o.N, o.prec);
  }
};
std::mutex g_tune_mu;
std::map<LeafKey, int> g_tuned;  // best leaf per bucket, this process

double wall() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct fde_batch_s {
  std::vector<fde_runner_t> r;
  std::vector<int> leaf;
  std::vector<cudaStream_t> streams;
  int device = 0;
  double setup_s = 0.0, tune_s = 0.0, solve_s = 0.0;
  long long instance_steps = 0;
  ~fde_batch_s() {
    for (auto x : r) fde_runner_free(x);
    for (auto s : streams) cudaStreamDestroy(s);
  }
};

using namespace fde;

static fde_runner_t make_runner(const fde_run_params& p, int leaf, const double* U0, cudaStream_t st,
                                fde_status* status) {
  fde_run_params q = p;
  q.op_x.leaf = leaf;
  q.op_y.leaf = leaf;
  fde_runner_t r = nullptr;
  *status = fde_runner_create(&q, U0, st, &r);
  return r;
}

// Time `steps` steps of a fresh runner with the given leaf; returns the runner.
static fde_runner_t trial(const fde_run_params& p, int leaf, const double* U0, cudaStream_t st, double* secs,
                          fde_status* status) {
  fde_runner_t r = make_runner(p, leaf, U0, st, status);
  if (*status != FDE_OK) return nullptr;
  const int warm = 1, steps = p.dim == 1 ? 4 : 2;
  *status = fde_runner_advance(r, warm, st);
  if (*status == FDE_OK) {
    const double t0 = wall();
    *status = fde_runner_advance(r, steps, st);  // synchronises the stream
    *secs = (wall() - t0) / steps;
  }
  if (*status != FDE_OK) {
    fde_runner_free(r);
    return nullptr;
  }
  return r;
}

extern "C" fde_status fde_batch_create(const fde_run_params* params, const double* const* U0, int count,
                                       const fde_batch_opts* opts, void* stream, fde_batch_t* out) {
  FDE_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  FDE_ARG(params != nullptr && U0 != nullptr && count >= 1, "bad instance arrays");
  const int threads = opts ? opts->threads : 4;
  const int autotune = opts ? opts->autotune : 0;
  FDE_ARG(threads >= 1 && threads <= 64, "threads must be in [1, 64]");
  for (int i = 0; i < count; ++i) FDE_ARG(U0[i] != nullptr, "NULL initial state");
  cudaStream_t st = (cudaStream_t)stream;
  fde_batch_s* B = new fde_batch_s();
  const double t0 = wall();
  auto fail = [&](fde_status s) {
    delete B;
    return s;
  };
  if (cudaGetDevice(&B->device) != cudaSuccess) return fail(FDE_ERR_CUDA);
  for (int t = 0; t < threads; ++t) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("fde_batch_create: stream creation failed");
      return fail(FDE_ERR_CUDA);
    }
    B->streams.push_back(s);
  }
  for (int i = 0; i < count; ++i) {
    const fde_run_params& p = params[i];
    const int N = p.op_x.N;
    fde_status s = FDE_OK;
    fde_runner_t r = nullptr;
    int leaf = p.op_x.leaf;
    if (autotune) {
      const LeafKey key{p.dim, N, p.prec};
      int cached = 0;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) cached = it->second;
      }
      if (cached) {
        leaf = cached;
      } else {
        // candidates: leaf sizes that give at least two leaves (a 1-leaf tree is plain dense)
        const int cands1[] = {32, 64, 128, 256}, cands2[] = {64, 128, 256};
        const int* c = p.dim == 1 ? cands1 : cands2;
        const int nc = p.dim == 1 ? 4 : 3;
        const double ts = wall();
        double best = 1e300;
        fde_runner_t keep = nullptr;
        int best_leaf = 0;
        for (int k = 0; k < nc; ++k) {
          if (c[k] * 2 > N && best_leaf) continue;
          double secs = 0.0;
          fde_runner_t tr = trial(p, c[k], U0[i], st, &secs, &s);
          if (!tr) return fail(s);
          if (secs < best) {
            if (keep) fde_runner_free(keep);
            keep = tr;
            best = secs;
            best_leaf = c[k];
          } else {
            fde_runner_free(tr);
          }
        }
        leaf = best_leaf;
        // the kept trial runner restarts from U0 (its statistics keep the trial steps)
        s = fde_runner_load(keep, U0[i], 0, st);
        if (s != FDE_OK) {
          fde_runner_free(keep);
          return fail(s);
        }
        r = keep;
        B->tune_s += wall() - ts;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = leaf;
      }
    }
    if (!r) {
      r = make_runner(p, leaf, U0[i], st, &s);
      if (!r) return fail(s);
    }
    B->r.push_back(r);
    B->leaf.push_back(leaf);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(FDE_ERR_CUDA);
  B->setup_s = wall() - t0;
  *out = B;
  return FDE_OK;
}

extern "C" fde_status fde_batch_advance(fde_batch_t b, int nsteps) {
  FDE_ARG(b != nullptr, "batch is NULL");
  FDE_ARG(nsteps >= 0, "nsteps must be >= 0");
  const int T = (int)b->streams.size(), n = (int)b->r.size();
  std::vector<fde_status> st(T, FDE_OK);
  std::vector<std::string> msg(T);
  const double t0 = wall();
  auto work = [&](int t) {
    if (cudaSetDevice(b->device) != cudaSuccess) {
      st[t] = FDE_ERR_CUDA;
      msg[t] = "cudaSetDevice failed in a batch worker";
      return;
    }
    for (int i = t; i < n; i += T) {
      const fde_status s = fde_runner_advance(b->r[i], nsteps, b->streams[t]);
      if (s != FDE_OK) {
        st[t] = s;
        msg[t] = std::string("instance ") + std::to_string(i) + ": " + fde_last_error();
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();
  b->solve_s += wall() - t0;
  for (int t = 0; t < T; ++t)
    if (st[t] != FDE_OK) {
      set_error("fde_batch_advance: %s", msg[t].c_str());
      return st[t];
    }
  b->instance_steps += (long long)nsteps * n;
  return FDE_OK;
}

extern "C" fde_status fde_batch_state(fde_batch_t b, int i, double* U_out, void* stream) {
  FDE_ARG(b != nullptr && U_out != nullptr, "NULL argument");
  FDE_ARG(i >= 0 && i < (int)b->r.size(), "instance index out of range");
  return fde_runner_state(b->r[i], U_out, stream);
}

extern "C" fde_status fde_batch_info(fde_batch_t b, int i, int* leaf, fde_run_stats* stats) {
  FDE_ARG(b != nullptr, "batch is NULL");
  FDE_ARG(i >= 0 && i < (int)b->r.size(), "instance index out of range");
  if (leaf) *leaf = b->leaf[i];
  if (stats) FDE_TRY(fde_runner_stats(b->r[i], stats));
  return FDE_OK;
}

extern "C" fde_status fde_batch_timing(fde_batch_t b, double* setup_s, double* tune_s, double* solve_s,
                                       long long* instance_steps) {
  FDE_ARG(b != nullptr, "batch is NULL");
  if (setup_s) *setup_s = b->setup_s;
  if (tune_s) *tune_s = b->tune_s;
  if (solve_s) *solve_s = b->solve_s;
  if (instance_steps) *instance_steps = b->instance_steps;
  return FDE_OK;
}

extern "C" void fde_batch_free(fde_batch_t b) { delete b; }
