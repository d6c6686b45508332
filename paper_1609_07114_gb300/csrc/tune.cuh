// Autotuner of the launch configuration (fdtd_autotune).  Included by
// fdtd.cu after the planners and the march.
//
// Every choice below leaves the results bit for bit unchanged (the kernels
// share one operation sequence per update; the model map's row and GEMM forms
// add in the same order), so only time is at stake:
//   - one or two steps per launch (FDTD_TB),
//   - the one-step tile height, or the row-marching kernel's resident CTAs
//     per SM (4 or 3), tile height, and how many rows it stages ahead
//     through shared memory or prefetches into L1,
//   - where the models' maps run on the two-step path (fused in the zone
//     tiles, or in the zone chain: every model, or the shared maps),
//   - from how many sharing simulations a map runs as a GEMM, and the GEMM
//     CTA shape (rows per warp).
// The search is one pass of coordinate descent from the fixed rule, in that
// order; each candidate is re-planned, marched warm-up + K steps from the
// current state (with the source and probe positions of the context's most
// recent run, the sources at zero amplitude) with the K steps timed by CUDA
// events on the context's stream, and the state restored from a device
// snapshot.
// A candidate replaces the best only if it is faster by more than 1% (graph
// replays repeat to a fraction of that).  The winner is kept for the
// context's life and, when a cache file is given, stored under a key of the
// device (name, SM count, clock), the grids and the embedded models' sizes, so
// that the next context of the same shape takes it without timing.

namespace {

struct TuneCfg {
  int tb_mode, chain, th1, thm, gmin, rpw, ring, pf, mb;
};

// The one-step tile table and per-simulation tile offsets on the device.
int upload_tiles(fdtd_ctx* ctx) {
  cudaFree(ctx->tiles_d);
  ctx->tiles_d = nullptr;
  CK(cudaMalloc(&ctx->tiles_d, sizeof(TileWork) * ctx->tiles.size()));
  CK(cudaMemcpy(ctx->tiles_d, ctx->tiles.data(), sizeof(TileWork) * ctx->tiles.size(), cudaMemcpyHostToDevice));
  std::vector<int> tb(ctx->sims.size() + 1);
  for (size_t s = 0; s < ctx->sims.size(); ++s) tb[s] = ctx->sims[s].tile_base;
  tb[ctx->sims.size()] = (int)ctx->tiles.size();
  CK(cudaMemcpy(ctx->tile_base_d, tb.data(), sizeof(int) * tb.size(), cudaMemcpyHostToDevice));
  return FDTD_OK;
}

int apply_cfg(fdtd_ctx* ctx, const TuneCfg& c) {
  ctx->tb_mode = c.tb_mode;
  ctx->tb_chain_mode = c.chain;
  ctx->ov_th1 = c.th1;
  ctx->ov_thm = c.thm;
  ctx->ov_gemm_min = c.gmin;
  ctx->ov_rpw = c.rpw;
  ctx->ov_ring = c.ring;
  ctx->ov_pf = c.pf;
  ctx->ov_mb = c.mb;
  drop_graphs(ctx);
  plan_tiles(ctx);
  int rc = upload_tiles(ctx);
  if (rc) return rc;
  return upload_instances(ctx);   // shared-map groups, then the two-step plan
}

// Device copy of the marching state: the current fields of every
// simulation, every model's [y; x~], the PML auxiliaries, the DFT sums.
struct TuneSnap {
  DevBuf<char> buf;
  std::vector<std::pair<void*, size_t>> parts;
  long long step = 0;
  int cur = 0;
  ~TuneSnap() { buf.release(); }
};

int snap_take(fdtd_ctx* ctx, TuneSnap& sn) {
  sn.parts.clear();
  const int c = ctx->cur;
  for (SimHost& sh : ctx->sims) {
    const size_t bytes = sizeof(float) * (size_t)(sh.ny + 1) * sh.pitch;
    sn.parts.push_back({sh.ex[c], bytes});
    sn.parts.push_back({sh.ey[c], bytes});
    sn.parts.push_back({sh.hz[c], bytes});
  }
  for (Instance& in : ctx->insts) sn.parts.push_back({in.state_d[c], sizeof(float) * (size_t)in.n});
  if (!ctx->pml_cells.empty())
    sn.parts.push_back({ctx->pml_psi.p, sizeof(float) * (2 * ctx->pml_cells.size() + ctx->pml_edges.size())});
  if (ctx->dft_nmon > 0) sn.parts.push_back({ctx->dft_acc.p, sizeof(double2) * (size_t)ctx->dft_nmon * ctx->dft_nfreq});
  size_t total = 0;
  for (auto& p : sn.parts) total += (p.second + 255) & ~(size_t)255;
  CK(sn.buf.reserve(total));
  size_t off = 0;
  for (auto& p : sn.parts) {
    CK(cudaMemcpyAsync(sn.buf.p + off, p.first, p.second, cudaMemcpyDeviceToDevice, ctx->stream));
    off += (p.second + 255) & ~(size_t)255;
  }
  sn.step = ctx->step;
  sn.cur = c;
  return FDTD_OK;
}

int snap_restore(fdtd_ctx* ctx, const TuneSnap& sn) {
  size_t off = 0;
  for (auto& p : sn.parts) {
    CK(cudaMemcpyAsync(p.first, sn.buf.p + off, p.second, cudaMemcpyDeviceToDevice, ctx->stream));
    off += (p.second + 255) & ~(size_t)255;
  }
  ctx->step = sn.step;
  ctx->cur = sn.cur;
  return FDTD_OK;
}

// Device ms per time step of the applied configuration over K steps (after
// `warm` untimed ones); the state is restored afterwards.
// The most recent run's sources (sharing one zero waveform, so the fields do
// not change) and probes (into a scratch buffer): the candidates are timed
// with the source and probe lists they will run with.
struct TuneRun {
  std::vector<fdtd_source> src;
  std::vector<const float*> wv;
  DevBuf<float> zero, pout;
  ~TuneRun() {
    zero.release();
    pout.release();
  }
};
constexpr int kTuneMaxSteps = kChunk + 512;   // warm-up + timed steps of one candidate

int tune_run_init(fdtd_ctx* ctx, TuneRun& tr) {
  tr.src = ctx->last_src;
  if (!tr.src.empty()) {
    CK(tr.zero.reserve(kTuneMaxSteps));
    CK(cudaMemsetAsync(tr.zero.p, 0, sizeof(float) * kTuneMaxSteps, ctx->stream));
    for (fdtd_source& s : tr.src) s.wave = tr.zero.p;
  }
  tr.wv.assign(std::max<size_t>(tr.src.size(), 1), tr.zero.p);
  if (!ctx->last_prb.empty()) CK(tr.pout.reserve((size_t)kTuneMaxSteps * ctx->last_prb.size()));
  return FDTD_OK;
}

int time_cfg(fdtd_ctx* ctx, const TuneSnap& sn, const TuneRun& tr, int warm, int K, double* ms) {
  const int nprobe = (int)ctx->last_prb.size();
  int rc = prepare_run(ctx, warm + K, tr.src.empty() ? nullptr : tr.src.data(), (int)tr.src.size(), tr.wv.data(),
                       nprobe ? ctx->last_prb.data() : nullptr, nprobe, tr.pout.p);
  if (rc) return rc;
  rc = march(ctx, warm, nprobe);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, ctx->stream));
  rc = march(ctx, K, nprobe);
  CK(cudaEventRecord(e1, ctx->stream));
  CK(cudaEventSynchronize(e1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *ms = (double)t / K;
  rc = snap_restore(ctx, sn);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

// Key of a context's tuning problem: device, grids, models (per simulation
// their sizes and which map they share, not their positions), layers,
// monitors.
std::string tune_key(const fdtd_ctx* ctx) {
  int dev = 0, nsm = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  std::string k = std::string(prop.name) + "|sm" + std::to_string(nsm) + "|khz" + std::to_string(clk);
  for (const SimHost& sh : ctx->sims)
    k += "|g" + std::to_string(sh.nx) + "x" + std::to_string(sh.ny) + (sh.all_dense ? "d" : "s");
  std::vector<const CoupledMap*> maps;
  for (const Instance& in : ctx->insts) {
    size_t m = 0;
    while (m < maps.size() && maps[m] != in.map.get()) ++m;
    if (m == maps.size()) maps.push_back(in.map.get());
    k += "|m" + std::to_string(in.sim) + "," + std::to_string(in.n) + "," + std::to_string(in.map->ld) + "," +
         std::to_string(m);
  }
  k += "|pml" + std::to_string(ctx->pml_cells.size()) + "|dft" + std::to_string(ctx->dft_nmon);
  uint64_t h = 1469598103934665603ull;   // FNV-1a
  for (unsigned char ch : k) h = (h ^ ch) * 1099511628211ull;
  char buf[32];
  snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, TuneCfg* c) {
  FILE* f = path ? fopen(path, "r") : nullptr;
  if (!f) return false;
  char line[256];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char k[64];
    TuneCfg t{};
    if (sscanf(line, "%63s tb=%d chain=%d th1=%d thm=%d gmin=%d rpw=%d ring=%d pf=%d mb=%d", k, &t.tb_mode,
               &t.chain, &t.th1, &t.thm, &t.gmin, &t.rpw, &t.ring, &t.pf, &t.mb) == 10 &&
        key == k) {
      *c = t;   // the last entry of a key wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const TuneCfg& c, double ms) {
  FILE* f = path ? fopen(path, "a") : nullptr;
  if (!f) return;
  fprintf(f, "%s tb=%d chain=%d th1=%d thm=%d gmin=%d rpw=%d ring=%d pf=%d mb=%d ms_per_step=%.6f\n", key.c_str(),
          c.tb_mode, c.chain, c.th1, c.thm, c.gmin, c.rpw, c.ring, c.pf, c.mb, ms);
  fclose(f);
}

void fill_report(const fdtd_ctx* ctx, fdtd_tune_report* rep) {
  if (!rep) return;
  rep->steps_per_launch = ctx->tb ? 2 : 1;
  rep->tile_rows = ctx->sims.empty() ? 0 : ctx->sims[0].th;
  rep->march_rows = ctx->tb && ctx->tb_march ? ctx->tbm_th : 0;
  rep->gemm_min = ctx->ov_gemm_min;
  rep->gemm_rows_per_warp = ctx->ov_rpw;
  rep->chain = ctx->tb_chain_mode;
  rep->march_ring = ctx->tb && ctx->tb_march ? ctx->tbm_ring : 0;
  rep->march_prefetch = ctx->tb && ctx->tb_march && ctx->tbm_ring == 0 ? ctx->tbm_pf : 0;
  rep->chained_models = ctx->tb ? ctx->tb_nchain : 0;
  rep->march_ctas = ctx->tb && ctx->tb_march ? ctx->tbm_mb : 0;
}

int run_autotune(fdtd_ctx* ctx, const char* cache_path, fdtd_tune_report* rep) {
  if (rep) *rep = fdtd_tune_report{};
  const char* path = cache_path ? cache_path : getenv("FDTD_TUNE_CACHE");
  if (path && !*path) path = nullptr;
  const std::string key = tune_key(ctx);
  TuneCfg cached;
  if (cache_lookup(path, key, &cached)) {
    int rc = apply_cfg(ctx, cached);
    if (rc) return rc;
    fill_report(ctx, rep);
    return FDTD_OK;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  TuneSnap sn;
  int rc = snap_take(ctx, sn);
  if (rc) return rc;
  TuneRun tr;
  rc = tune_run_init(ctx, tr);
  if (rc) return rc;
  // the fixed rule (as the context was created), then per dimension
  bool shared = false;   // some map is used by two or more instances
  for (size_t a = 0; a < ctx->insts.size() && !shared; ++a)
    for (size_t b = a + 1; b < ctx->insts.size() && !shared; ++b)
      shared = ctx->insts[a].map == ctx->insts[b].map;
  TuneCfg best{ctx->tb_mode, ctx->tb_chain_mode, 0, 0, 0, 0, -1, kNoOverride, 0};
  rc = apply_cfg(ctx, best);
  if (rc) return rc;
  double t_def = 0;
  rc = time_cfg(ctx, sn, tr, kChunk, kChunk, &t_def);
  if (rc) return rc;
  // K: a multiple of the graph chunk lasting a few ms
  const int K = std::max(kChunk, std::min(512, (int)std::ceil(4.0 / std::max(t_def, 1e-4) / kChunk) * kChunk));
  rc = time_cfg(ctx, sn, tr, kChunk, K, &t_def);
  if (rc) return rc;
  double t_best = t_def;
  int ncand = 2;
  auto tryc = [&](TuneCfg c) -> int {
    int r = apply_cfg(ctx, c);
    if (r) return r;
    if (c.tb_mode == 1 && !ctx->tb) return FDTD_OK;   // the two-step path does not apply here
    double t = 0;
    r = time_cfg(ctx, sn, tr, kChunk, K, &t);
    if (r) return r;
    ++ncand;
    if (t < 0.99 * t_best) t_best = t, best = c;
    return FDTD_OK;
  };
  rc = apply_cfg(ctx, best);
  if (rc) return rc;
  best.tb_mode = ctx->tb ? 1 : 0;   // the fixed rule's choice (timed above), pinned
  {
    // the other path; two steps also with each placement of the models'
    // maps (fused tiles, the zone chain for every model or the shared maps)
    TuneCfg c = best;
    c.tb_mode = 1 - best.tb_mode;
    if ((rc = tryc(c))) return rc;
    if (!ctx->insts.empty())
      for (int ch : {-1, 0, 1}) {
        TuneCfg d = best;
        d.tb_mode = 1;
        d.chain = ch;
        if (d.tb_mode == best.tb_mode && d.chain == best.chain) continue;
        if ((rc = tryc(d))) return rc;
      }
  }
  {
    rc = apply_cfg(ctx, best);
    if (rc) return rc;
    const bool two = ctx->tb;
    const int cand1[] = {16, 24, 32, 48, 64, 96, 128};
    const int cand2[] = {8, 16, 24, 32, 48, 64, 96, 128, 192, 256};
    if (two) {
      {   // 3 resident CTAs per SM (more registers per thread, loads in registers)
        TuneCfg c = best;
        c.mb = 3;
        if ((rc = tryc(c))) return rc;
      }
      for (int th : cand2) {
        TuneCfg c = best;
        c.thm = th;
        if ((rc = tryc(c))) return rc;
      }
      for (int rg : {0, 2, 3, 4}) {
        if (best.mb == 3) break;   // that form loads into registers only
        TuneCfg c = best;
        c.ring = rg;
        if ((rc = tryc(c))) return rc;
      }
      for (int p : {0, -1, -2, -3}) {   // rows prefetched into L1 ahead of the register loads
        TuneCfg c = best;
        c.pf = p;
        if ((rc = tryc(c))) return rc;
      }
      if (!ctx->insts.empty())
        for (int ch : {-1, 0, 1}) {
          if (ch == best.chain) continue;
          TuneCfg c = best;
          c.chain = ch;
          if ((rc = tryc(c))) return rc;
        }
    } else {
      for (int th : cand1) {
        TuneCfg c = best;
        c.th1 = th;
        if ((rc = tryc(c))) return rc;
      }
    }
  }
  if (shared) {
    for (int g : {1, 1 << 30}) {
      TuneCfg c = best;
      c.gmin = g;
      if ((rc = tryc(c))) return rc;
    }
    rc = apply_cfg(ctx, best);
    if (rc) return rc;
    if (ctx->ngwork > 0)
      for (int r : {1, 2}) {
        TuneCfg c = best;
        c.rpw = r;
        if ((rc = tryc(c))) return rc;
      }
  }
  rc = apply_cfg(ctx, best);
  if (rc) return rc;
  rc = snap_restore(ctx, sn);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  cache_store(path, key, best, t_best);
  fill_report(ctx, rep);
  if (rep) {
    rep->candidates = ncand;
    rep->ms_default = t_def;
    rep->ms_best = t_best;
  }
  return FDTD_OK;
}

}  // namespace
