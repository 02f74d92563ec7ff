// Several PT-CN systems stepped together (pt_batch_*; include/pt.h).
//
// The paper batches the pair FFTs of one system into library calls (Sec. 3.2).
// Here the pair tiles of all systems of a batch go into the same launch groups:
// round r of the tile tournament of every system forms one merged round (no
// two tiles of a round share an output orbital, within or across systems), so
// small systems, whose own launch groups leave most of the GPU idle, share each
// pair-kernel launch. The merged pair-kernel sequence is captured once into a
// CUDA graph and replayed every step. Every tile carries the addresses of its
// own system's orbitals and accumulators, and each W element receives its tile
// contributions in the same order as in the system's own exchange, so a batched
// system's results are bitwise those of the same system stepped alone with the
// same pair tile.
//
// A batch step interleaves the systems' PT-CN phases (engine.cu): every system
// runs on its own stream; the SCF iterations are enqueued for all systems that
// have not converged before any density change is read, so the systems' kernels
// overlap on the device; the exchange of the new orbitals is the merged launch
// sequence on the batch's stream, ordered against the systems' streams by events.
#include <climits>

#include "engine.h"

struct pt_batch {
  std::vector<pt_system*> sys;
  cudaStream_t s = nullptr;
  int tile = 0, tpl = 0;
  Grid3 gf{};
  bool mixed = false;
  const void* khat = nullptr;          // kernel table of the first system (all are equal)
  pt::DevTwiddles tw{};
  pt::FockPlan plan{};                 // merged tiles (device copy in the batch workspace)
  void* X = nullptr;                   // pair intermediate of one launch group
  std::vector<cudaEvent_t> ev_sys;
  cudaEvent_t ev_batch = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int runs = 0;                        // merged exchanges so far (the graph is captured after the first)
  long long graph_kernels = 0;
  bool timing = false;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  double pair_ms = 0.0;
  long long pairs = 0, groups = 0;
  std::string err;
};

namespace {

constexpr int kMaxBatch = 1024;

pt_status batch_fail(pt_batch* b, const std::string& msg, pt_status st) {
  if (b) b->err = msg;
  g_last_error = msg;
  return st;
}

// The systems can share pair launches when their pair FFTs use the same grid, precision,
// kernel table (cell, screening, mixing) and basis (which fixes the axis-2 reach).
bool compatible(const pt_system* a, const pt_system* b, std::string* why) {
  const pt_params &p = a->p, &q = b->p;
  if (a->gf.n0 != b->gf.n0 || a->gf.n1 != b->gf.n1 || a->gf.n2 != b->gf.n2 || a->g.n0 != b->g.n0 ||
      a->g.n1 != b->g.n1 || a->g.n2 != b->g.n2) { *why = "grids differ"; return false; }
  if (a->mixed != b->mixed) { *why = "precisions differ"; return false; }
  for (int k = 0; k < 3; ++k)
    if (p.cell[k] != q.cell[k]) { *why = "cells differ"; return false; }
  if (p.omega != q.omega || p.alpha != q.alpha || p.ecut != q.ecut) { *why = "kernel or cutoff differs"; return false; }
  if (p.alpha == 0.0) { *why = "no exchange (alpha = 0)"; return false; }
  return true;
}

// Merged schedule: the tournament rounds of every system (tiles bound to that system's
// orbitals and accumulators), round r of all systems together, split into launch groups
// of at most tpl tiles. Returns the host tiles and launch lists; `count_only` sizes it.
struct Merged {
  std::vector<pt::PairTile> tiles;
  std::vector<int> first, count;
  int max_group = 0;
};

pt_status merge_schedule(const std::vector<pt_system*>& sys, int tile, int tpl, Merged* out, std::string* why) {
  std::vector<std::vector<std::vector<pt::PairTile>>> rounds(sys.size());
  size_t nr = 0;
  for (size_t i = 0; i < sys.size(); ++i) {
    pt::PairTile* t = nullptr;
    int *lf = nullptr, *lc = nullptr, nl = 0;
    const int nt = pt::fock_build_tiles(sys[i]->ne, 0, tile, 1, INT_MAX, &t, &lf, &lc, &nl);
    if (nt < 0) { *why = "tile schedule"; return PT_ERR_INVALID; }
    pt::fock_bind_tiles(t, nt, fock_orbitals_addr(sys[i]), nullptr, sys[i]->w_r, nullptr, sys[i]->Nf,
                        exchange_cs(sys[i]));
    for (int l = 0; l < nl; ++l) rounds[i].emplace_back(t + lf[l], t + lf[l] + lc[l]);   // one launch = one round
    std::free(t); std::free(lf); std::free(lc);
    nr = std::max(nr, rounds[i].size());
  }
  out->tiles.clear(); out->first.clear(); out->count.clear(); out->max_group = 0;
  for (size_t r = 0; r < nr; ++r) {
    std::vector<pt::PairTile> rd;
    for (size_t i = 0; i < sys.size(); ++i)
      if (r < rounds[i].size()) rd.insert(rd.end(), rounds[i][r].begin(), rounds[i][r].end());
    for (size_t k = 0; k < rd.size(); k += (size_t)tpl) {
      const int cnt = (int)std::min<size_t>((size_t)tpl, rd.size() - k);
      out->first.push_back((int)out->tiles.size());
      out->count.push_back(cnt);
      out->max_group = std::max(out->max_group, cnt);
      out->tiles.insert(out->tiles.end(), rd.begin() + k, rd.begin() + k + cnt);
    }
  }
  return PT_OK;
}

int batch_tile(const std::vector<pt_system*>& sys, int pair_tile) {
  if (pair_tile > 0) return pair_tile;
  int mx = 1;
  for (auto* s : sys) mx = std::max(mx, s->ne);
  return std::min(pt::kTileMax, mx);
}

// tiles per launch group: as asked, else a whole merged round (the largest is the round of
// diagonal tiles, one per orbital block of every system) up to a 16 GB pair intermediate
int batch_tpl(const std::vector<pt_system*>& sys, int tile, int tiles_per_launch) {
  long round_max = 0;
  for (auto* s : sys) round_max += (s->ne + tile - 1) / tile;
  const double per_tile = (double)pt::kTileMax * pt::kTileMax * sys[0]->Nf * exchange_cs(sys[0]);
  const long cap = (long)std::max(1.0, std::floor(16.0e9 / per_tile));
  long tpl = std::min(round_max, cap);
  if (tiles_per_launch > 0) tpl = std::min<long>(tpl, tiles_per_launch);
  return (int)std::max<long>(1, tpl);
}

pt_status check_systems(pt_system* const* systems, int nsys, std::vector<pt_system*>* out, std::string* why) {
  if (systems == nullptr || nsys < 1 || nsys > kMaxBatch) { *why = "need 1 <= nsys <= 1024 systems"; return PT_ERR_INVALID; }
  out->assign(systems, systems + nsys);
  for (int i = 0; i < nsys; ++i) {
    if ((*out)[i] == nullptr) { *why = "NULL system"; return PT_ERR_INVALID; }
    for (int j = 0; j < i; ++j)
      if ((*out)[j] == (*out)[i]) { *why = "a system appears twice"; return PT_ERR_INVALID; }
    std::string w;
    if (!compatible((*out)[0], (*out)[i], &w)) { *why = "system " + std::to_string(i) + ": " + w; return PT_ERR_INVALID; }
  }
  return PT_OK;
}

size_t batch_layout(const Merged& m, int tpl, const pt_system* s0, uintptr_t base, pt::PairTile** tiles, void** X) {
  Carver c{base};
  pt::PairTile* t = c.take<pt::PairTile>(std::max<size_t>(1, m.tiles.size()));
  void* x = c.take<unsigned char>((size_t)tpl * pt::kTileMax * pt::kTileMax * s0->Nf * exchange_cs(s0));
  if (tiles) *tiles = t;
  if (X) *X = x;
  return c.off + 256;
}

pt_status pair_launches(pt_batch* b) {
  if (b->mixed)
    return pt::fock_pairs<float>(b->plan, 1, b->gf, (const float*)b->khat, b->X, b->tw, b->s) == cudaSuccess
               ? PT_OK : PT_ERR_CUDA;
  return pt::fock_pairs<double>(b->plan, 1, b->gf, (const double*)b->khat, b->X, b->tw, b->s) == cudaSuccess
             ? PT_OK : PT_ERR_CUDA;
}

// W = V_X Psi of every system's current orbitals (real-space orbitals current) into out[i]
pt_status batch_exchange_run(pt_batch* b, double2* const* out) {
  const size_t n = b->sys.size();
  for (size_t i = 0; i < n; ++i) {
    pt_system* sys = b->sys[i];
    pt_status st = exchange_prepare(sys, sys->psi);
    if (st != PT_OK) return batch_fail(b, "system " + std::to_string(i) + ": " + sys->err, st);
    if (cudaEventRecord(b->ev_sys[i], sys->s) != cudaSuccess || cudaStreamWaitEvent(b->s, b->ev_sys[i], 0) != cudaSuccess)
      return batch_fail(b, "batch: event ordering failed", PT_ERR_CUDA);
  }
  if (b->timing && cudaEventRecord(b->t0, b->s) != cudaSuccess) return batch_fail(b, "batch: timing event", PT_ERR_CUDA);
  if (b->runs == 0) {
    // first run: direct launches (they also set the kernels' one-time attributes); then
    // capture the same sequence into a graph for every later run
    if (pair_launches(b) != PT_OK) return batch_fail(b, "batch: pair kernels -> " + pt::cuda_msg(cudaGetLastError()), PT_ERR_CUDA);
  } else {
    if (b->exec == nullptr) {
      const unsigned long long before = pt::launch_count();
      cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const pt_status ps = pair_launches(b);
        e = cudaStreamEndCapture(b->s, &b->graph);
        if (ps != PT_OK && e == cudaSuccess) e = cudaErrorUnknown;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      b->graph_kernels = (long long)(pt::launch_count() - before);
      pt::launched(-(int)b->graph_kernels);   // capturing launches nothing
      if (e != cudaSuccess) return batch_fail(b, "batch: graph capture -> " + pt::cuda_msg(e), PT_ERR_CUDA);
    }
    if (cudaGraphLaunch(b->exec, b->s) != cudaSuccess) return batch_fail(b, "batch: graph launch", PT_ERR_CUDA);
    pt::launched((int)b->graph_kernels);
  }
  b->runs += 1;
  if (b->timing) {
    float ms = 0.f;
    if (cudaEventRecord(b->t1, b->s) != cudaSuccess || cudaEventSynchronize(b->t1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, b->t0, b->t1) != cudaSuccess)
      return batch_fail(b, "batch: timing event", PT_ERR_CUDA);
    b->pair_ms += ms;
    for (auto* sys : b->sys) b->pairs += (long long)sys->ne * (sys->ne + 1) / 2;
    b->groups += b->plan.n_launch;
  }
  if (cudaEventRecord(b->ev_batch, b->s) != cudaSuccess) return batch_fail(b, "batch: event ordering failed", PT_ERR_CUDA);
  for (size_t i = 0; i < n; ++i) {
    pt_system* sys = b->sys[i];
    if (cudaStreamWaitEvent(sys->s, b->ev_batch, 0) != cudaSuccess) return batch_fail(b, "batch: event ordering failed", PT_ERR_CUDA);
    pt_status st = exchange_finish(sys, out[i], 0);
    if (st != PT_OK) return batch_fail(b, "system " + std::to_string(i) + ": " + sys->err, st);
  }
  return PT_OK;
}

}  // namespace

extern "C" {

pt_status pt_batch_workspace_size(pt_system* const* systems, int nsys, int pair_tile, int tiles_per_launch,
                                  size_t* bytes) {
  std::vector<pt_system*> sys;
  std::string why;
  pt_status st = check_systems(systems, nsys, &sys, &why);
  if (st != PT_OK) return batch_fail(nullptr, "pt_batch_workspace_size: " + why, st);
  if (bytes == nullptr || pair_tile < 0 || pair_tile > pt::kTileMax || tiles_per_launch < 0)
    return batch_fail(nullptr, "pt_batch_workspace_size: NULL output, pair_tile outside [0, 4] or tiles_per_launch < 0",
                      PT_ERR_INVALID);
  const int tile = batch_tile(sys, pair_tile);
  const int tpl = batch_tpl(sys, tile, tiles_per_launch);
  Merged m;
  st = merge_schedule(sys, tile, tpl, &m, &why);
  if (st != PT_OK) return batch_fail(nullptr, "pt_batch_workspace_size: " + why, st);
  *bytes = batch_layout(m, tpl, sys[0], 0, nullptr, nullptr);
  return PT_OK;
}

pt_status pt_batch_create(pt_system* const* systems, int nsys, int pair_tile, int tiles_per_launch, void* d_ws,
                          size_t ws_bytes, void* stream, pt_batch** out) {
  const char* fn = "pt_batch_create: ";
  std::vector<pt_system*> sys;
  std::string why;
  pt_status st = check_systems(systems, nsys, &sys, &why);
  if (st != PT_OK) return batch_fail(nullptr, fn + why, st);
  if (out == nullptr || d_ws == nullptr || ((uintptr_t)d_ws & 255) != 0 || pair_tile < 0 || pair_tile > pt::kTileMax ||
      tiles_per_launch < 0 || stream == nullptr)
    return batch_fail(nullptr, std::string(fn) + "NULL output, workspace or stream, workspace not 256-byte aligned, "
                      "or bad tile", PT_ERR_INVALID);
  pt_batch* b = new pt_batch();
  b->sys = sys;
  b->s = (cudaStream_t)stream;
  b->tile = batch_tile(sys, pair_tile);
  b->tpl = batch_tpl(sys, b->tile, tiles_per_launch);
  b->gf = sys[0]->gf;
  b->mixed = sys[0]->mixed;
  b->khat = b->mixed ? (const void*)sys[0]->khat32 : (const void*)sys[0]->khat64;
  b->tw = sys[0]->tw;
  Merged m;
  st = merge_schedule(sys, b->tile, b->tpl, &m, &why);
  if (st != PT_OK) { delete b; return batch_fail(nullptr, fn + why, st); }
  const size_t need = batch_layout(m, b->tpl, sys[0], 0, nullptr, nullptr);
  if (ws_bytes < need) {
    delete b;
    return batch_fail(nullptr, std::string(fn) + "workspace too small (" + std::to_string(need) + " bytes needed)",
                      PT_ERR_OOM);
  }
  pt::PairTile* d_tiles = nullptr;
  batch_layout(m, b->tpl, sys[0], (uintptr_t)d_ws, &d_tiles, &b->X);
  cudaError_t e = cudaMemcpyAsync(d_tiles, m.tiles.data(), sizeof(pt::PairTile) * m.tiles.size(),
                                  cudaMemcpyHostToDevice, b->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
  b->plan.tile = b->tile;
  b->plan.tiles_per_launch = b->tpl;
  b->plan.n_launch = (int)m.first.size();
  b->plan.launch_first = (int*)std::malloc(sizeof(int) * std::max<size_t>(1, m.first.size()));
  b->plan.launch_count = (int*)std::malloc(sizeof(int) * std::max<size_t>(1, m.count.size()));
  std::copy(m.first.begin(), m.first.end(), b->plan.launch_first);
  std::copy(m.count.begin(), m.count.end(), b->plan.launch_count);
  b->plan.d_tiles = d_tiles;
  b->plan.n_tiles = (int)m.tiles.size();
  b->plan.g2_reach = sys[0]->plan_sym.g2_reach;   // the systems share cell and cutoff
  b->ev_sys.assign(sys.size(), nullptr);
  for (size_t i = 0; e == cudaSuccess && i < sys.size(); ++i) e = cudaEventCreateWithFlags(&b->ev_sys[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_batch, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    const std::string msg = std::string(fn) + pt::cuda_msg(e);
    pt_batch_destroy(b);
    return batch_fail(nullptr, msg, PT_ERR_CUDA);
  }
  *out = b;
  return PT_OK;
}

pt_status pt_batch_exchange(pt_batch* b, void* const* d_w) {
  if (b == nullptr || d_w == nullptr) return batch_fail(b, "pt_batch_exchange: NULL batch or outputs", PT_ERR_INVALID);
  std::vector<double2*> out(b->sys.size());
  for (size_t i = 0; i < out.size(); ++i) {
    if (d_w[i] == nullptr) return batch_fail(b, "pt_batch_exchange: NULL output", PT_ERR_INVALID);
    out[i] = (double2*)d_w[i];
    pt_system* sys = b->sys[i];
    if (!sys->psi_r_current) {
      pt_status st = real_orbitals(sys, sys->psi);
      if (st != PT_OK) return batch_fail(b, "system " + std::to_string(i) + ": " + sys->err, st);
      sys->psi_r_current = true;
    }
  }
  pt_status st = batch_exchange_run(b, out.data());
  if (st != PT_OK) return st;
  for (auto* sys : b->sys)
    if (cudaStreamSynchronize(sys->s) != cudaSuccess) return batch_fail(b, "pt_batch_exchange: synchronisation", PT_ERR_CUDA);
  return PT_OK;
}

pt_status pt_batch_step(pt_batch* b, pt_step_info* out_host) {
  if (b == nullptr) return batch_fail(nullptr, "pt_batch_step: NULL batch", PT_ERR_INVALID);
  const size_t n = b->sys.size();
  std::vector<StepCtx> c(n);
  auto fail = [&](size_t i, pt_status st) { return batch_fail(b, "system " + std::to_string(i) + ": " + b->sys[i]->err, st); };
  for (size_t i = 0; i < n; ++i) {
    const pt_status st = cn_begin(b->sys[i], &c[i]);
    if (st != PT_OK) return fail(i, st);
  }
  // SCF iterations: enqueue one for every system still iterating, then read their
  // density changes (each read waits for its own stream only); a system whose SCF is
  // done may restart it after an outer ACE rebuild (ace_outer)
  for (bool any = true; any;) {
    for (size_t i = 0; i < n; ++i)
      if (!c[i].done) {
        const pt_status st = cn_iterate(b->sys[i], &c[i]);
        if (st != PT_OK) return fail(i, st);
      }
    any = false;
    for (size_t i = 0; i < n; ++i)
      if (!c[i].done) {
        pt_status st = cn_check(b->sys[i], &c[i]);
        bool again = false;
        if (st == PT_OK && c[i].done) st = cn_outer(b->sys[i], &c[i], &again);
        if (st != PT_OK) return fail(i, st);
        any = any || !c[i].done;
      }
  }
  for (size_t i = 0; i < n; ++i) {
    const pt_status st = cn_orthonormalize(b->sys[i], &c[i]);
    if (st != PT_OK) return fail(i, st);
  }
  std::vector<double2*> out(n);
  for (size_t i = 0; i < n; ++i) out[i] = b->sys[i]->wg;
  pt_status st = batch_exchange_run(b, out.data());
  if (st != PT_OK) return st;
  pt_status worst = PT_OK;
  for (size_t i = 0; i < n; ++i) {
    pt_step_info info{};
    const pt_status si = cn_complete(b->sys[i], &c[i], &info);
    if (out_host) out_host[i] = info;
    if (si == PT_ERR_NOT_CONVERGED) { worst = si; continue; }
    if (si != PT_OK) return fail(i, si);
  }
  return worst;
}

pt_status pt_batch_set_timing(pt_batch* b, int enable) {
  if (b == nullptr) return batch_fail(nullptr, "pt_batch_set_timing: NULL batch", PT_ERR_INVALID);
  if (enable && b->t0 == nullptr) {
    if (cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess)
      return batch_fail(b, "pt_batch_set_timing: event creation failed", PT_ERR_CUDA);
  }
  b->timing = enable != 0;
  return PT_OK;
}

pt_status pt_batch_get_timing(pt_batch* b, double* pair_ms, int64_t* pairs, int64_t* launch_groups, int reset) {
  if (b == nullptr) return batch_fail(nullptr, "pt_batch_get_timing: NULL batch", PT_ERR_INVALID);
  if (pair_ms) *pair_ms = b->pair_ms;
  if (pairs) *pairs = b->pairs;
  if (launch_groups) *launch_groups = b->groups;
  if (reset) { b->pair_ms = 0.0; b->pairs = 0; b->groups = 0; }
  return PT_OK;
}

pt_status pt_batch_destroy(pt_batch* b) {
  if (b == nullptr) return PT_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->ev_sys)
    if (e) cudaEventDestroy(e);
  if (b->ev_batch) cudaEventDestroy(b->ev_batch);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  std::free(b->plan.launch_first);
  std::free(b->plan.launch_count);
  delete b;
  return PT_OK;
}

}  // extern "C"
