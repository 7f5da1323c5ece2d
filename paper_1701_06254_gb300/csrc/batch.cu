// An ensemble of independent reservoir models advanced together on one GPU.
//
// Every member is an ordinary simulator (its own state, Jacobian, RAS
// factors, AMG hierarchy and Krylov basis) bound to a stream of its own.  A
// pool of host worker threads takes members largest-first and runs each one's
// time loop; while one member's host thread waits on its stream (the
// residual estimate after every Arnoldi step), the others keep the GPU fed,
// so many small systems that would each leave most of the 152 SMs idle share
// the device.  Members never exchange data: each one's results are exactly
// those of the same model run alone, whatever the worker count.
//
// The worker count is the tuning knob.  sim_batch_autotune tries candidate
// counts on the largest members for one time step each, keeps the fastest,
// and puts every member's state and statistics back as they were.
#include "common.cuh"
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <memory>
#include <thread>

struct sim_batch_s {
  int dev = 0;
  int workers = 8;
  std::vector<sim_t> member;
  std::vector<cudaStream_t> stream;
  std::vector<int> order;            // members by decreasing cell count (longest first)
  std::vector<long long> cells;
  ~sim_batch_s() {
    for (sim_t m : member) if (m) sim_destroy(m);
    for (cudaStream_t s : stream) if (s) cudaStreamDestroy(s);
  }
};

#define ABI_BEGIN try {
#define ABI_END                                                       \
  }                                                                   \
  catch (const rs_error &e) { return e.code; }                        \
  catch (const std::bad_alloc &) { rs_set_error("host allocation failed"); return SIM_ERR_OOM; } \
  catch (...) { rs_set_error("unexpected exception"); return SIM_ERR_CUDA; }                       \
  return SIM_OK;

extern "C" sim_status sim_batch_create(sim_batch_t *out, int n_members, const sim_grid *grids, const sim_rock *rocks,
                                       const sim_fluid *fluids, const sim_well *const *wells, const int *n_wells,
                                       const sim_options *opts, int n_workers) {
  ABI_BEGIN
  if (!out || n_members < 1 || !grids || !rocks || !fluids || !wells || !n_wells || !opts || n_workers < 0)
    RS_FAIL(SIM_ERR_ARG, "sim_batch_create: bad argument");
  *out = nullptr;
  for (int k = 0; k < n_members; k++)
    if (const char *e = rs_opts_invalid(&opts[k])) RS_FAIL(SIM_ERR_ARG, "sim_batch_create: member %d: %s", k, e);
  std::unique_ptr<sim_batch_s> b(new sim_batch_s());
  RS_CUDA(cudaGetDevice(&b->dev));
  b->workers = n_workers > 0 ? n_workers : 8;
  b->member.assign(n_members, nullptr);
  b->stream.assign(n_members, nullptr);
  b->cells.resize(n_members);
  for (int k = 0; k < n_members; k++) {
    RS_CUDA(cudaStreamCreateWithFlags(&b->stream[k], cudaStreamNonBlocking));
    sim_options o = opts[k];
    o.cuda_stream = b->stream[k];
    sim_status rc = sim_create(&b->member[k], &grids[k], &rocks[k], &fluids[k], wells[k], n_wells[k], &o);
    if (rc != SIM_OK) {
      std::string msg = sim_last_error();
      RS_FAIL(rc, "sim_batch_create: member %d: %s", k, msg.c_str());
    }
    b->cells[k] = (long long)grids[k].nx * grids[k].ny * grids[k].nz;
  }
  b->order.resize(n_members);
  for (int k = 0; k < n_members; k++) b->order[k] = k;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return b->cells[a] > b->cells[c]; });
  *out = b.release();
  ABI_END
}

extern "C" void sim_batch_destroy(sim_batch_t b) { delete b; }

extern "C" sim_status sim_batch_member(sim_batch_t b, int k, sim_t *member) {
  ABI_BEGIN
  if (!b || !member || k < 0 || k >= (int)b->member.size()) RS_FAIL(SIM_ERR_ARG, "sim_batch_member: bad argument");
  *member = b->member[k];
  ABI_END
}

extern "C" sim_status sim_batch_size(sim_batch_t b, int *n_members, int *n_workers) {
  ABI_BEGIN
  if (!b) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  if (n_members) *n_members = (int)b->member.size();
  if (n_workers) *n_workers = b->workers;
  ABI_END
}

// Advances the members listed in idx by n_steps each with w worker threads.
// Per-member statuses and error texts go to st[] / msg[] (indexed by member).
static void run_members(sim_batch_s *b, const std::vector<int> &idx, int n_steps, int w, sim_stats *stats,
                        std::vector<sim_status> &st, std::vector<std::string> &msg) {
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(b->dev);
    for (;;) {
      int q = next.fetch_add(1);
      if (q >= (int)idx.size()) break;
      int k = idx[q];
      sim_stats s;
      st[k] = sim_advance(b->member[k], n_steps, &s);
      if (st[k] != SIM_OK) msg[k] = sim_last_error();
      if (stats) stats[k] = s;
    }
  };
  w = std::max(1, std::min(w, (int)idx.size()));
  std::vector<std::thread> pool;
  pool.reserve(w - 1);
  for (int t = 1; t < w; t++) pool.emplace_back(work);
  work();                                          // the calling thread is worker 0
  for (auto &t : pool) t.join();
}

extern "C" sim_status sim_batch_advance(sim_batch_t b, int n_steps, sim_stats *stats, sim_status *status) {
  ABI_BEGIN
  if (!b || n_steps < 0) RS_FAIL(SIM_ERR_ARG, "sim_batch_advance: bad argument");
  int m = (int)b->member.size();
  std::vector<sim_status> st(m, SIM_OK);
  std::vector<std::string> msg(m);
  run_members(b, b->order, n_steps, b->workers, stats, st, msg);
  if (status) for (int k = 0; k < m; k++) status[k] = st[k];
  for (int k = 0; k < m; k++)
    if (st[k] != SIM_OK) RS_FAIL(st[k], "member %d: %s", k, msg[k].c_str());
  ABI_END
}

// copy of one member's state and statistics, on the device
struct saved_member {
  dbuf<double> p, s, pb, y, sc;
  double t = 0.0;
  int have = 0;
  sim_stats stats;
};

static void save_member(sim_t h, saved_member &sv) {
  int n = 0, nw = 0;
  sim_stats s;
  if (sim_get_stats(h, &s) != SIM_OK) RS_FAIL(SIM_ERR_CUDA, "autotune: %s", sim_last_error());
  sv.stats = s;
  // sizes are fixed at creation; the state is read into device buffers
  sim_dims(h, &n, &nw);
  sv.p.ensure(n); sv.s.ensure(n); sv.pb.ensure(std::max(nw, 1));
  if (sim_get_state(h, sv.p.p, sv.s.p, nw ? sv.pb.p : nullptr, &sv.t) != SIM_OK)
    RS_FAIL(SIM_ERR_CUDA, "autotune: %s", sim_last_error());
  sv.y.ensure(4 * (size_t)(n + nw)); sv.sc.ensure(8);
  sv.have = sim_history(h, sv.y.p, sv.sc.p, 0, true);
}

static void restore_member(sim_t h, const saved_member &sv) {
  int n = 0, nw = 0;
  sim_dims(h, &n, &nw);
  if (sim_set_state(h, sv.p.p, sv.s.p, nw ? sv.pb.p : nullptr, sv.t) != SIM_OK)
    RS_FAIL(SIM_ERR_CUDA, "autotune: %s", sim_last_error());
  sim_put_stats(h, &sv.stats);
  sim_history(h, sv.y.p, sv.sc.p, sv.have, false);
}

extern "C" sim_status sim_batch_autotune(sim_batch_t b, const int *candidates, int n_candidates, int sample,
                                         int *chosen, double *seconds) {
  ABI_BEGIN
  if (!b || !candidates || n_candidates < 1) RS_FAIL(SIM_ERR_ARG, "sim_batch_autotune: bad argument");
  for (int c = 0; c < n_candidates; c++)
    if (candidates[c] < 1) RS_FAIL(SIM_ERR_ARG, "sim_batch_autotune: worker counts must be positive");
  int m = (int)b->member.size();
  int maxw = *std::max_element(candidates, candidates + n_candidates);
  if (sample < 1) sample = std::min(m, 2 * maxw);
  sample = std::min(sample, m);
  std::vector<int> idx(b->order.begin(), b->order.begin() + sample);
  std::vector<saved_member> sv(sample);
  for (int q = 0; q < sample; q++) save_member(b->member[idx[q]], sv[q]);
  int best = b->workers;
  double best_t = 1e300;
  std::vector<sim_status> st(m, SIM_OK);
  std::vector<std::string> msg(m);
  for (int c = 0; c < n_candidates; c++) {
    RS_CUDA(cudaDeviceSynchronize());
    auto t0 = std::chrono::steady_clock::now();
    run_members(b, idx, 1, candidates[c], nullptr, st, msg);
    RS_CUDA(cudaDeviceSynchronize());
    double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (seconds) seconds[c] = dt;
    for (int q = 0; q < sample; q++) restore_member(b->member[idx[q]], sv[q]);
    for (int q = 0; q < sample; q++)
      if (st[idx[q]] != SIM_OK) RS_FAIL(st[idx[q]], "autotune: member %d: %s", idx[q], msg[idx[q]].c_str());
    if (dt < best_t) { best_t = dt; best = candidates[c]; }
  }
  RS_CUDA(cudaDeviceSynchronize());
  b->workers = best;
  if (chosen) *chosen = best;
  ABI_END
}
