// Batched solves of independent sequences: the k-points of one self-consistent cycle each
// give their own sequence of pencils (Section 1), with uneven sizes.  A batch owns several
// contexts, each with its own stream, and runs one host worker thread per context; the
// workers take whole sequences from a shared counter, so that the host synchronisations and
// the latency-bound kernels of one sequence (Jacobi rounds, single-CTA factorisations, the
// per-loop read-backs) overlap the tensor-core products of another.
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

struct chfsi_batch {
  std::vector<chfsi_ctx*> ctx;
  int dev = 0;
  std::string err;
};

extern "C" {

int chfsi_batch_create(chfsi_batch** out, int32_t workers, int64_t n_max, int32_t blk_max,
                       const chfsi_opts* opts) {
  if (!out) return CHFSI_EINVAL;
  *out = nullptr;
  if (workers < 1 || workers > 64) return CHFSI_EINVAL;
  chfsi_opts o;
  chfsi_default_opts(&o);
  if (opts) o = *opts;
  o.cuda_stream = nullptr;  // every context creates and owns its stream
  auto* b = new chfsi_batch;
  if (cudaGetDevice(&b->dev) != cudaSuccess) {
    delete b;
    return CHFSI_ECUDA;
  }
  for (int w = 0; w < workers; ++w) {
    chfsi_ctx* c = nullptr;
    const int rc = chfsi_create(&c, n_max, blk_max, &o);
    if (rc != CHFSI_OK) {
      for (chfsi_ctx* x : b->ctx) chfsi_destroy(x);
      delete b;
      return rc;
    }
    b->ctx.push_back(c);
  }
  *out = b;
  return CHFSI_OK;
}

void chfsi_batch_destroy(chfsi_batch* b) {
  if (!b) return;
  for (chfsi_ctx* c : b->ctx) chfsi_destroy(c);
  delete b;
}

const char* chfsi_batch_last_error(const chfsi_batch* b) { return b ? b->err.c_str() : "null batch"; }

int chfsi_batch_solve(chfsi_batch* b, int32_t K, int32_t N, const int64_t* n, const int32_t* nev,
                      const int32_t* blk, int32_t deg, double tol, const chfsi_z* const* A,
                      const chfsi_z* const* B, const int64_t* ld, double* const* evals,
                      chfsi_z* const* evecs, chfsi_stats* st) {
  if (!b) return CHFSI_EINVAL;
  b->err.clear();
  if (K <= 0 || N <= 0 || !n || !nev || !blk || !A || !B || !ld || !evals) {
    b->err = "chfsi_batch_solve: bad arguments";
    return CHFSI_EINVAL;
  }
  for (int s = 0; s < K; ++s) {
    if (!evals[s] || ld[s] < n[s]) {
      b->err = "chfsi_batch_solve: bad arguments for sequence " + std::to_string(s);
      return CHFSI_EINVAL;
    }
  }
  std::atomic<int> next{0};
  std::atomic<int> first_rc{CHFSI_OK};
  std::mutex mu;
  auto work = [&](int w) {
    cudaSetDevice(b->dev);
    chfsi_ctx* c = b->ctx[w];
    for (;;) {
      if (first_rc.load() != CHFSI_OK) break;
      const int s = next.fetch_add(1);
      if (s >= K) break;
      int rc = chfsi_reset_warm_state(c);
      if (rc == CHFSI_OK)
        rc = chfsi_solve_sequence(c, N, n[s], A + (int64_t)s * N, B + (int64_t)s * N, ld[s], nullptr,
                                  nev[s], blk[s], deg, tol, evals[s], evecs ? evecs + (int64_t)s * N : nullptr,
                                  st ? st + (int64_t)s * N : nullptr);
      if (rc != CHFSI_OK) {
        std::lock_guard<std::mutex> g(mu);
        if (first_rc.load() == CHFSI_OK) {
          b->err = "sequence " + std::to_string(s) + ": " + chfsi_last_error(c);
          first_rc.store(rc);
        }
        break;
      }
    }
  };
  const int workers = (int)b->ctx.size();
  std::vector<std::thread> pool;
  for (int w = 1; w < std::min(workers, K); ++w) pool.emplace_back(work, w);
  work(0);
  for (std::thread& t : pool) t.join();
  return first_rc.load();
}

}  // extern "C"
