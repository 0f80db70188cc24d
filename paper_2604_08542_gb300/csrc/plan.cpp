// Host-side schedule of the chunk recurrence.
//
// A chain (sequence s, head h) carries its fast weights from chunk to chunk
// (Sec. 4.4: one GPU processes the chunks sequentially).  Chunk step j of a
// chain needs the weights W_j after j updates; at that step two independent
// sweeps over tokens use W_j:
//   - the gradient of chunk j at W_j (Eq. 8 is evaluated at the pre-chunk
//     weights), whose update produces W_{j+1};
//   - the apply of chunk j-1, whose queries see W_j, the weights after
//     chunk j-1's own update (Sec. 4.2).
// The planner lays every chain's step-j work side by side, cuts each token
// range into pieces so that one step fills the GPU (longest pieces first),
// and gives every gradient piece a slot for its partial sum; because the
// chunk gradient is a plain sum over tokens (Eq. 8, Eq. 10), the pieces'
// partial sums add up to it, in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>

#include "ttt_internal.h"

namespace scal3r {

namespace {

constexpr size_t kScratchTileBytes = 3 * 32 * 1024;   // BF16 backward: three 128x128 bf16 images per tile

struct Task {
  int32_t chain, seq, role, chunk;
  int64_t t0, t1;
  float cost;
  int32_t wchunk;
};

// Cut [t0, t1) into n nearly equal pieces with boundaries on `align` tokens
// from t0 (the kernels' token tile).
std::vector<std::pair<int64_t, int64_t>> split(int64_t t0, int64_t t1, int n, int64_t align) {
  std::vector<std::pair<int64_t, int64_t>> out;
  int64_t len = t1 - t0;
  int64_t tiles = (len + align - 1) / align;
  if (n > tiles) n = (int)std::max<int64_t>(1, tiles);
  int64_t base = tiles / n, extra = tiles % n;
  int64_t cur = t0;
  for (int i = 0; i < n; ++i) {
    int64_t nt = base + (i < extra ? 1 : 0);
    int64_t end = std::min(t1, cur + nt * align);
    if (i == n - 1) end = t1;
    out.push_back({cur, end});
    cur = end;
  }
  return out;
}

// Pieces per task.  Every task starts with one piece; then, while the step
// has CTAs left, the task whose pieces are costliest gets one more.  This
// minimises the costliest piece (which sets the step's duration) without
// ever launching more pieces than CTAs.  A piece keeps at least one tile and
// min_tokens tokens.
std::vector<int> pieces_per_task(const std::vector<Task>& tasks, const Schedule& sch, int64_t ctas) {
  std::vector<int> n(tasks.size(), 1);
  std::priority_queue<std::pair<double, size_t>> heap;
  for (size_t i = 0; i < tasks.size(); ++i) heap.push({(double)tasks[i].cost, i});
  int64_t used = (int64_t)tasks.size();
  while (used < ctas && !heap.empty()) {
    const size_t i = heap.top().second;
    heap.pop();
    const int64_t len = tasks[i].t1 - tasks[i].t0;
    const int64_t tiles = (len + sch.align - 1) / sch.align;
    const int m = n[i] + 1;
    if (m > tiles || len / m < sch.min_tokens) continue;   // cannot be cut further
    n[i] = m;
    ++used;
    heap.push({(double)tasks[i].cost / m, i});
  }
  return n;
}

// ---- tail fill ------------------------------------------------------------
// With one wave of pieces, a task whose CTA share was rounded down keeps long
// pieces while the SMs of shorter pieces idle until the launch ends.  The fill
// caps every first-wave piece at a target time M and cuts the tokens that no
// longer fit into extra pieces placed behind the first wave.  A grid's CTA k
// starts on the first SM that frees once CTAs 0..k-1 are resident, so the
// extra pieces are sized, earliest first, for the modelled moments at which
// the first wave's SMs free.  M is the smallest target the model can meet
// (bisection); the fill is kept only if M beats the one-wave plan's modelled
// end by fill_margin.

struct Cut {
  int64_t t0, t1;
  bool fill;      // placed behind the first wave
  double start;   // modelled start of a fill piece
};

// A piece's modelled time.  The kernels run whole tiles (a ragged last tile
// costs a full one), so tokens count in tiles.
double fill_time(const Schedule& sch, int role, int64_t tokens) {
  const int64_t tiles = (tokens + sch.align - 1) / sch.align;
  const double t = (double)(tiles * sch.align);
  switch (role) {
    case ROLE_KEY: return sch.fill_ovh[0] + t * sch.fill_key_tok;
    case ROLE_APPLY: return sch.fill_ovh[1] + t;
    case ROLE_BKEY:
      return sch.fill_ovh[2] + t * sch.fill_bkey_tok +
             (double)((tiles + kBwdSubTiles - 1) / kBwdSubTiles) * sch.fill_bkey_sub;
    default: return sch.fill_ovh[3] + t;
  }
}

// The largest number of tiles (at most `avail` tiles, i.e. the tokens left
// from `t0` to `t1`) whose piece, started at `start`, ends by M; 0 if none.
int64_t tiles_by(const Schedule& sch, int role, int64_t t0, int64_t t1, double start, double M) {
  int64_t lo = 0, hi = (t1 - t0 + sch.align - 1) / sch.align;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    const int64_t tok = std::min(t1 - t0, mid * sch.align);
    if (start + fill_time(sch, role, tok) <= M) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Cuts of every task for target M (first-wave pieces: npieces[i] of them),
// or false if some tokens do not fit.
bool try_fill(const std::vector<Task>& tasks, const std::vector<int>& npieces, const Schedule& sch,
              int64_t ctas, double M, std::vector<std::vector<Cut>>& cuts) {
  cuts.assign(tasks.size(), {});
  std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
  std::vector<std::pair<double, size_t>> rest;   // (cost of the tokens left, task)
  std::vector<int64_t> next(tasks.size());
  int64_t first = 0;
  // The model prices each piece's fixed cost, so the fill's pieces are sized
  // by it alone, down to one tile (min_tokens governs the one-wave split).
  for (size_t i = 0; i < tasks.size(); ++i) {
    const Task& t = tasks[i];
    const int64_t tiles = (t.t1 - t.t0 + sch.align - 1) / sch.align;
    const int64_t cap = tiles_by(sch, t.role, t.t0, t.t1, 0.0, M);
    if (cap < 1) return false;
    const int64_t cov = std::min(tiles, (int64_t)npieces[i] * cap);
    const int64_t end = std::min(t.t1, t.t0 + cov * sch.align);
    for (auto& pr : split(t.t0, end, npieces[i], sch.align)) {
      cuts[i].push_back({pr.first, pr.second, false, 0.0});
      free_at.push(fill_time(sch, t.role, pr.second - pr.first));
      ++first;
    }
    next[i] = end;
    if (end < t.t1) rest.push_back({fill_time(sch, t.role, t.t1 - end), i});
  }
  // SMs the first wave leaves empty: their pieces start with it, at time 0
  for (int64_t k = first; k < ctas; ++k) free_at.push(-(double)sch.fill_start);
  std::stable_sort(rest.begin(), rest.end(),
                   [](const std::pair<double, size_t>& a, const std::pair<double, size_t>& b) {
                     return a.first > b.first;
                   });
  int64_t extra = 0;
  for (const auto& r : rest) {
    const Task& t = tasks[r.second];
    int64_t cur = next[r.second];
    while (cur < t.t1) {
      if (free_at.empty() || ++extra > ctas) return false;
      const double f = free_at.top() + sch.fill_start;
      free_at.pop();
      const int64_t n = tiles_by(sch, t.role, cur, t.t1, f, M);
      if (n < 1) return false;
      const int64_t e = std::min(t.t1, cur + n * sch.align);
      cuts[r.second].push_back({cur, e, true, f});
      free_at.push(f + fill_time(sch, t.role, e - cur));
      cur = e;
    }
  }
  return true;
}

// Cuts of every task: the one-wave split, or the fill when it pays.
std::vector<std::vector<Cut>> cut_tasks(const std::vector<Task>& tasks, const std::vector<int>& npieces,
                                        const Schedule& sch, int64_t ctas, bool fill) {
  std::vector<std::vector<Cut>> one(tasks.size());
  double m1 = 0.0, work = 0.0;
  int64_t total = 0;
  for (size_t i = 0; i < tasks.size(); ++i) {
    for (auto& pr : split(tasks[i].t0, tasks[i].t1, npieces[i], sch.align)) {
      one[i].push_back({pr.first, pr.second, false, 0.0});
      const double c = fill_time(sch, tasks[i].role, pr.second - pr.first);
      m1 = std::max(m1, c);
      work += c;
    }
    total += npieces[i];
  }
  if (!fill || total > ctas || tasks.empty()) return one;
  std::vector<std::vector<Cut>> best, trial;
  double lo = work / (double)ctas, hi = m1;
  for (int it = 0; it < 48 && hi - lo > 0.5; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (try_fill(tasks, npieces, sch, ctas, mid, trial)) {
      hi = mid;
      best.swap(trial);
    } else {
      lo = mid;
    }
  }
  if (best.empty() || hi > m1 * (1.0 - sch.fill_margin)) return one;
  return best;
}

void lay_out_step(const std::vector<Task>& tasks, const Schedule& sch, int num_sms, int waves,
                  bool backward, std::vector<WorkItem>& items, std::vector<UpdateItem>& upds,
                  std::vector<Step>& steps, int32_t& max_slots,
                  const std::vector<UpdateItem>& step_updates_template) {
  Step st{};
  st.item0 = (int32_t)items.size();
  st.upd0 = (int32_t)upds.size();
  int ctas = sch.ctas_per_wave > 0 ? sch.ctas_per_wave : num_sms;
  const std::vector<int> npieces = pieces_per_task(tasks, sch, std::max<int64_t>(1, (int64_t)waves * ctas));
  const bool fill = waves == 1 && (sch.fill & (backward ? 2 : 1)) != 0;
  const std::vector<std::vector<Cut>> cuts = cut_tasks(tasks, npieces, sch, ctas, fill);
  // pieces per task; a piece's modelled start orders the fill pieces
  std::vector<WorkItem> step_items;
  std::vector<Cut> where;
  // slots: per chain, slots are contiguous (key pieces, and in the backward
  // also apply pieces, of the same chain), in token order.
  std::vector<UpdateItem> upd = step_updates_template;
  int32_t slot = 0;
  for (auto& u : upd) {
    u.slot0 = slot;
    u.nslots = 0;
    for (size_t ti = 0; ti < tasks.size(); ++ti) {
      const Task& t = tasks[ti];
      if (t.chain != u.chain) continue;
      bool reduces = backward || t.role == ROLE_KEY;
      if (!reduces) continue;
      for (const Cut& c : cuts[ti]) {
        WorkItem w{c.t0, c.t1, t.chain, t.role, slot++, t.seq, t.wchunk, 0};
        step_items.push_back(w);
        where.push_back(c);
        u.nslots++;
      }
    }
  }
  for (size_t ti = 0; ti < tasks.size(); ++ti) {
    const Task& t = tasks[ti];
    bool reduces = backward || t.role == ROLE_KEY;
    if (reduces) continue;
    for (const Cut& c : cuts[ti]) {
      WorkItem w{c.t0, c.t1, t.chain, t.role, -1, t.seq, t.wchunk, 0};
      step_items.push_back(w);
      where.push_back(c);
    }
  }
  // the first wave, longest (costliest) pieces first; then the fill pieces by
  // modelled start (a negative start: an SM the first wave left empty)
  auto cost_of = [&](const WorkItem& w) {
    double c = (double)(w.t1 - w.t0);
    if (w.role == ROLE_KEY) c *= sch.key_cost;
    if (w.role == ROLE_BKEY) c *= sch.bkey_cost;
    return c;
  };
  std::vector<size_t> order(step_items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    const bool fa = where[a].fill, fb = where[b].fill;
    if (fa != fb) return fb;
    if (fa) return where[a].start < where[b].start;
    return cost_of(step_items[a]) > cost_of(step_items[b]);
  });
  {
    std::vector<WorkItem> sorted;
    sorted.reserve(order.size());
    for (size_t i : order) {
      sorted.push_back(step_items[i]);
      if (where[i].fill) st.nfill++;
    }
    step_items.swap(sorted);
  }
  if (backward) {
    // one sub-piece of scratch and a weight image per update-VJP piece (BF16
    // backward; the apply-VJP pieces keep their factors in shared memory)
    int32_t tiles = 0;
    for (auto& w : step_items) {
      w.aux = tiles;
      if (w.role == ROLE_BKEY) tiles += kBwdScratchTiles;
    }
    st.scratch_tiles = tiles;
  }
  items.insert(items.end(), step_items.begin(), step_items.end());
  upds.insert(upds.end(), upd.begin(), upd.end());
  st.nitems = (int32_t)step_items.size();
  st.nupd = (int32_t)upd.size();
  st.nslots = slot;
  max_slots = std::max(max_slots, slot);
  steps.push_back(st);
}

}  // namespace

int build_plan(Plan& plan, const Shape& s, const Schedule& sch_in, int num_sms,
               const int64_t* off, int32_t C, const int32_t* ptr, int32_t S, int32_t ckpt_every,
               bool mse_compose) {
  // the composed squared-error loss launches part of each backward step
  // separately, outside the fill's one-launch model
  Schedule sch = sch_in;
  if (mse_compose) sch.fill = 0;
  if (!off || !ptr || C < 0 || S < 1) return SCAL3R_ERR_INVALID_ARG;
  if (off[0] != 0) return SCAL3R_ERR_INVALID_ARG;
  for (int32_t c = 0; c < C; ++c)
    if (off[c + 1] <= off[c]) return SCAL3R_ERR_INVALID_ARG;  // empty or decreasing chunk
  if (ptr[0] != 0 || ptr[S] != C) return SCAL3R_ERR_INVALID_ARG;
  for (int32_t i = 0; i < S; ++i)
    if (ptr[i + 1] < ptr[i]) return SCAL3R_ERR_INVALID_ARG;
  if (C > 0 && off[C] > ((int64_t)1 << 40)) return SCAL3R_ERR_INVALID_ARG;

  Plan p;
  p.chunk_offsets.assign(off, off + C + 1);
  p.seq_chunk_ptr.assign(ptr, ptr + S + 1);
  p.H = s.H;
  p.S = S;
  p.C = C;
  p.T = off[C];
  int32_t maxn = 0;
  for (int32_t i = 0; i < S; ++i) maxn = std::max(maxn, ptr[i + 1] - ptr[i]);
  p.max_chunks = maxn;
  const int32_t H = s.H;
  // checkpoints: with n = ckpt_every > 1 only the weights after local chunks
  // n-1, 2n-1, ... are stored, sequence after sequence
  const int32_t nck = ckpt_every > 1 ? ckpt_every : 1;
  p.ckpt_every = nck;
  p.mse_compose = mse_compose;
  std::vector<int64_t> cbase(S, 0);
  for (int32_t q = 1; q < S; ++q) cbase[q] = cbase[q - 1] + (ptr[q] - ptr[q - 1]) / nck;
  p.ckpt_slots = cbase[S - 1] + (ptr[S] - ptr[S - 1]) / nck;
  // where the backward reads W_j of sequence q (j >= 1): its checkpoint, or
  // (sparse, j not a multiple of n) the recompute buffer at the chain's row
  auto wsrc = [&](int32_t q, int32_t j) -> int32_t {
    if (j == 0) return -1;
    if (nck == 1) return ptr[q] + j - 1;
    if (j % nck == 0) return (int32_t)(cbase[q] + j / nck - 1);
    return q;
  };

  // ---- forward: steps j = 0 .. maxn --------------------------------------
  for (int32_t j = 0; j <= maxn; ++j) {
    std::vector<Task> tasks;
    std::vector<UpdateItem> upd;
    for (int32_t q = 0; q < S; ++q) {
      int32_t n = ptr[q + 1] - ptr[q];
      if (j > n) continue;
      for (int32_t h = 0; h < H; ++h) {
        int32_t chain = q * H + h;
        if (j < n) {
          int32_t c = ptr[q] + j;
          tasks.push_back({chain, q, ROLE_KEY, c, off[c], off[c + 1],
                           (float)(off[c + 1] - off[c]) * sch.key_cost, -1});
          UpdateItem u{};
          u.chain = chain;
          u.chunk = c;
          u.last = (j == n - 1);
          u.seq = q;
          u.wslot = nck == 1 ? c : ((j + 1) % nck == 0 ? (int32_t)(cbase[q] + (j + 1) / nck - 1) : -1);
          upd.push_back(u);
        }
        if (j >= 1) {
          int32_t c = ptr[q] + j - 1;
          tasks.push_back({chain, q, ROLE_APPLY, c, off[c], off[c + 1], (float)(off[c + 1] - off[c]), -1});
        }
        if (n == 0 && j == 0) {
          UpdateItem u{};
          u.chain = chain;
          u.chunk = -1;   // no chunk: w_final = w0
          u.last = 1;
          u.seq = q;
          u.wslot = -1;
          upd.push_back(u);
        }
      }
    }
    lay_out_step(tasks, sch, num_sms, sch.fwd_waves, false, p.items, p.updates, p.steps, p.max_slots, upd);
    if (mse_compose) {   // the residual pieces: the gradient pieces' ranges, as apply pieces
      const Step& fs = p.steps.back();
      Step ys{};
      ys.item0 = (int32_t)p.yitems.size();
      for (int32_t i = fs.item0; i < fs.item0 + fs.nitems; ++i)
        if (p.items[i].role == ROLE_KEY) {
          WorkItem y = p.items[i];
          y.role = ROLE_APPLY;
          y.slot = -1;
          p.yitems.push_back(y);
        }
      ys.nitems = (int32_t)p.yitems.size() - ys.item0;
      p.ysteps.push_back(ys);
    }
  }

  // ---- backward: steps j = maxn .. 0 -------------------------------------
  for (int32_t j = maxn; j >= 0; --j) {
    std::vector<Task> tasks;
    std::vector<UpdateItem> upd;
    for (int32_t q = 0; q < S; ++q) {
      int32_t n = ptr[q + 1] - ptr[q];
      if (n == 0 || j > n) continue;
      for (int32_t h = 0; h < H; ++h) {
        int32_t chain = q * H + h;
        if (j < n) {
          int32_t c = ptr[q] + j;
          tasks.push_back({chain, q, ROLE_BKEY, c, off[c], off[c + 1],
                           (float)(off[c + 1] - off[c]) * sch.bkey_cost, wsrc(q, j)});
          if (mse_compose)
            tasks.push_back({chain, q, ROLE_BAPPLY_K, c, off[c], off[c + 1], (float)(off[c + 1] - off[c]),
                             wsrc(q, j)});
        }
        if (j >= 1) {
          int32_t c = ptr[q] + j - 1;
          tasks.push_back({chain, q, ROLE_BAPPLY, c, off[c], off[c + 1], (float)(off[c + 1] - off[c]), wsrc(q, j)});
        }
        UpdateItem u{};
        u.chain = chain;
        u.chunk = (j >= 1) ? ptr[q] + j - 1 : -1;   // the update whose norm VJP follows
        u.last = (j == n);                           // no adjoint from a later chunk yet
        u.first = (j == 0);
        u.seq = q;
        u.wslot = wsrc(q, j);
        upd.push_back(u);
      }
    }
    lay_out_step(tasks, sch, num_sms, sch.bwd_waves, true, p.bitems, p.bupdates, p.bsteps, p.bmax_slots, upd);
    p.bscratch_tiles = std::max<int64_t>(p.bscratch_tiles, p.bsteps.back().scratch_tiles);
    Step& bs = p.bsteps.back();
    if (mse_compose) {   // the key-side apply VJPs last: they run after the update VJPs
      auto first = p.bitems.begin() + bs.item0;
      auto mid = std::stable_partition(first, first + bs.nitems,
                                       [](const WorkItem& w) { return w.role != ROLE_BAPPLY_K; });
      bs.npost = (int32_t)(first + bs.nitems - mid);
    }
    if (nck > 1 && j % nck != 0) {
      bs.wseg = j % nck;
      if (j == maxn || (j + 1) % nck == 0) {   // the segment's last step comes first: recompute it
        bs.rec0 = j - j % nck;
        bs.nrec = j % nck;
        bs.segk = j / nck;
      }
    }
  }

  // ---- sparse checkpoints: forward steps to rerun, segment sources --------
  if (nck > 1) {
    for (int32_t j = 0; j < maxn; ++j) {
      const Step& fs = p.steps[j];
      Step rs{};
      rs.item0 = (int32_t)p.ritems.size();
      rs.upd0 = (int32_t)p.rupdates.size();
      for (int32_t i = fs.item0; i < fs.item0 + fs.nitems; ++i)
        if (p.items[i].role == ROLE_KEY) p.ritems.push_back(p.items[i]);
      for (int32_t i = fs.upd0; i < fs.upd0 + fs.nupd; ++i) {
        UpdateItem u = p.updates[i];
        if (u.chunk < 0) continue;
        u.wslot = u.seq;   // the recompute buffer's row of the chain
        u.last = 0;
        p.rupdates.push_back(u);
      }
      rs.nitems = (int32_t)p.ritems.size() - rs.item0;
      rs.nupd = (int32_t)p.rupdates.size() - rs.upd0;
      rs.nslots = fs.nslots;
      p.rsteps.push_back(rs);
    }
    for (int32_t k = 0; k * nck <= maxn; ++k)
      for (int32_t q = 0; q < S; ++q) {
        const int32_t n = ptr[q + 1] - ptr[q];
        p.segsrc.push_back(k * nck > n ? -2 : (k == 0 ? -1 : (int32_t)(cbase[q] + k - 1)));
      }
  }
  p.valid = true;
  plan = std::move(p);
  return SCAL3R_OK;
}

size_t workspace_bytes(const Plan& p, const Shape& s, bool with_backward) {
  const size_t chains = (size_t)p.S * s.H;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t b = 0;
  b += al(2 * chains * s.P() * sizeof(float));                  // wm
  b += al(chains * s.R() * sizeof(float));                      // rho
  size_t slots = std::max(p.max_slots, with_backward ? p.bmax_slots : 0);
  b += al(std::max<size_t>(slots, 1) * s.P() * sizeof(float));  // partials
  if (with_backward) {
    b += al(chains * s.P() * sizeof(float));                    // rbuf
    b += al(chains * s.R() * sizeof(float));                    // drho
    b += al(chains * s.P() * sizeof(float));                    // dw0 per chain
    b += al((size_t)p.bscratch_tiles * kScratchTileBytes + 1024);   // BF16 backward scratch
    if (p.ckpt_every > 1) b += al((size_t)(p.ckpt_every - 1) * chains * s.P() * sizeof(float));   // wseg
  }
  if (p.mse_compose) {   // residuals (and the backward's key-side dk), bf16 [T][H][D]
    const size_t tok = al((size_t)p.T * s.H * s.D * 2);
    b += tok * (with_backward ? 2 : 1);
  }
  return b;
}

void carve_workspace(const Plan& p, const Shape& s, bool with_backward, void* ws, Params& prm) {
  const size_t chains = (size_t)p.S * s.H;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* c = (char*)ws;
  prm.wm = (float*)c;
  c += al(2 * chains * s.P() * sizeof(float));
  prm.rho = (float*)c;
  c += al(chains * s.R() * sizeof(float));
  prm.part = (float*)c;
  size_t slots = std::max(p.max_slots, with_backward ? p.bmax_slots : 0);
  c += al(std::max<size_t>(slots, 1) * s.P() * sizeof(float));
  if (with_backward) {
    prm.rbuf = (float*)c;
    c += al(chains * s.P() * sizeof(float));
    prm.drho = (float*)c;
    c += al(chains * s.R() * sizeof(float));
    prm.dw0_chain = (float*)c;
    c += al(chains * s.P() * sizeof(float));
    prm.scratch = (void*)(((uintptr_t)c + 1023) & ~(uintptr_t)1023);
    prm.scratch_tiles = p.bscratch_tiles;
    c += al((size_t)p.bscratch_tiles * kScratchTileBytes + 1024);
    prm.wseg = p.ckpt_every > 1 ? (float*)c : nullptr;
    if (p.ckpt_every > 1) c += al((size_t)(p.ckpt_every - 1) * chains * s.P() * sizeof(float));
  } else {
    prm.wseg = nullptr;
    prm.rbuf = prm.drho = prm.dw0_chain = nullptr;
    prm.scratch = nullptr;
    prm.scratch_tiles = 0;
  }
  prm.rtok = prm.dk2 = nullptr;
  if (p.mse_compose) {
    const size_t tok = al((size_t)p.T * s.H * s.D * 2);
    prm.rtok = (void*)c;
    c += tok;
    if (with_backward) prm.dk2 = (void*)c;
  }
}

}  // namespace scal3r
