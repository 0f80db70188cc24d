// Test harness around the host-side chunk-step planner (csrc/plan.cpp).
//
// The planner is plain host C++; the tests compile it with this file into a
// small shared library and read the plan back through these C calls, so its
// invariants are checked on a machine without a GPU.  Nothing here is part of
// the product library.
#include <cstdint>
#include <cstring>

#include "../paper_2604_08542_gb300/csrc/ttt_internal.h"

using scal3r::Plan;
using scal3r::Schedule;
using scal3r::Shape;

extern "C" {

// Build a plan.  sched = {ctas_per_wave, fwd_waves, bwd_waves, min_tokens,
// align, fill}, costs = {key_cost, bkey_cost}; ckpt_every and mse_compose as the
// library passes them (sparse checkpoints; the composed squared-error loss of
// the BF16 head_dim-64 path).  Returns the plan (or null) and the planner's
// status in *rc.
void* ph_build_opts(int32_t H, int32_t D, int32_t F, int32_t num_sms, const int32_t* sched, const float* costs,
                    const int64_t* off, int32_t C, const int32_t* ptr, int32_t S, int32_t ckpt_every,
                    int32_t mse_compose, int32_t* rc) {
  Schedule sch;
  sch.ctas_per_wave = sched[0];
  sch.fwd_waves = sched[1];
  sch.bwd_waves = sched[2];
  sch.min_tokens = sched[3];
  sch.align = sched[4];
  sch.fill = sched[5];
  sch.key_cost = costs[0];
  sch.bkey_cost = costs[1];
  Shape s{H, D, F};
  Plan* p = new Plan();
  *rc = scal3r::build_plan(*p, s, sch, num_sms, off, C, ptr, S, ckpt_every, mse_compose != 0);
  if (*rc != 0) {
    delete p;
    return nullptr;
  }
  return p;
}


void ph_free(void* p) { delete (Plan*)p; }

// out = {items, updates, steps, max_slots, bitems, bupdates, bsteps,
//        bmax_slots, bscratch_tiles, max_chunks}
void ph_counts(const void* pv, int64_t* out) {
  const Plan& p = *(const Plan*)pv;
  out[0] = (int64_t)p.items.size();
  out[1] = (int64_t)p.updates.size();
  out[2] = (int64_t)p.steps.size();
  out[3] = p.max_slots;
  out[4] = (int64_t)p.bitems.size();
  out[5] = (int64_t)p.bupdates.size();
  out[6] = (int64_t)p.bsteps.size();
  out[7] = p.bmax_slots;
  out[8] = p.bscratch_tiles;
  out[9] = p.max_chunks;
}

// 8 values per piece: t0, t1, chain, role, slot, seq, wchunk, aux
void ph_items(const void* pv, int32_t backward, int64_t* out) {
  const Plan& p = *(const Plan*)pv;
  const auto& v = backward ? p.bitems : p.items;
  for (size_t i = 0; i < v.size(); ++i) {
    const scal3r::WorkItem& w = v[i];
    int64_t* o = out + 8 * i;
    o[0] = w.t0; o[1] = w.t1; o[2] = w.chain; o[3] = w.role;
    o[4] = w.slot; o[5] = w.seq; o[6] = w.wchunk; o[7] = w.aux;
  }
}

// 7 values per update: chain, chunk, slot0, nslots, last, seq, first
void ph_updates(const void* pv, int32_t backward, int32_t* out) {
  const Plan& p = *(const Plan*)pv;
  const auto& v = backward ? p.bupdates : p.updates;
  for (size_t i = 0; i < v.size(); ++i) {
    const scal3r::UpdateItem& u = v[i];
    int32_t* o = out + 7 * i;
    o[0] = u.chain; o[1] = u.chunk; o[2] = u.slot0; o[3] = u.nslots;
    o[4] = u.last; o[5] = u.seq; o[6] = u.first;
  }
}

// 6 values per step: item0, nitems, upd0, nupd, nslots, scratch_tiles
void ph_steps(const void* pv, int32_t backward, int32_t* out) {
  const Plan& p = *(const Plan*)pv;
  const auto& v = backward ? p.bsteps : p.steps;
  for (size_t i = 0; i < v.size(); ++i) {
    const scal3r::Step& s = v[i];
    int32_t* o = out + 6 * i;
    o[0] = s.item0; o[1] = s.nitems; o[2] = s.upd0; o[3] = s.nupd; o[4] = s.nslots; o[5] = s.scratch_tiles;
  }
}

int64_t ph_workspace(const void* pv, int32_t H, int32_t D, int32_t F, int32_t backward) {
  Shape s{H, D, F};
  return (int64_t)scal3r::workspace_bytes(*(const Plan*)pv, s, backward != 0);
}

// Carve a workspace of ph_workspace bytes starting at `base` and report each
// region's offset: wm, rho, part, rbuf, drho, dw0_chain, scratch (-1: none).
void ph_carve(const void* pv, int32_t H, int32_t D, int32_t F, int32_t backward, int64_t base, int64_t* out) {
  Shape s{H, D, F};
  scal3r::Params prm;
  std::memset(&prm, 0, sizeof(prm));
  scal3r::carve_workspace(*(const Plan*)pv, s, backward != 0, (void*)(uintptr_t)base, prm);
  const void* r[7] = {prm.wm, prm.rho, prm.part, prm.rbuf, prm.drho, prm.dw0_chain, prm.scratch};
  for (int i = 0; i < 7; ++i) out[i] = r[i] ? (int64_t)((uintptr_t)r[i] - (uintptr_t)base) : -1;
}

int32_t ph_bwd_scratch_tiles_per_piece() { return scal3r::kBwdScratchTiles; }

// out = {ritems, rupdates, rsteps, segsrc, yitems, ysteps, ckpt_slots, ckpt_every}
void ph_counts2(const void* pv, int64_t* out) {
  const Plan& p = *(const Plan*)pv;
  out[0] = (int64_t)p.ritems.size();
  out[1] = (int64_t)p.rupdates.size();
  out[2] = (int64_t)p.rsteps.size();
  out[3] = (int64_t)p.segsrc.size();
  out[4] = (int64_t)p.yitems.size();
  out[5] = (int64_t)p.ysteps.size();
  out[6] = p.ckpt_slots;
  out[7] = p.ckpt_every;
}

// The number of tail-fill pieces of every step (0: forward, 1: backward).
void ph_nfill(const void* pv, int32_t backward, int32_t* out) {
  const Plan& p = *(const Plan*)pv;
  const auto& v = backward ? p.bsteps : p.steps;
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].nfill;
}

// 5 values per backward step: wseg, rec0, nrec, segk, npost
void ph_bsteps2(const void* pv, int32_t* out) {
  const Plan& p = *(const Plan*)pv;
  for (size_t i = 0; i < p.bsteps.size(); ++i) {
    const scal3r::Step& s = p.bsteps[i];
    int32_t* o = out + 5 * i;
    o[0] = s.wseg; o[1] = s.rec0; o[2] = s.nrec; o[3] = s.segk; o[4] = s.npost;
  }
}

// The weight slot of every update (0: forward, 1: backward, 2: the recompute updates).
void ph_wslots(const void* pv, int32_t which, int32_t* out) {
  const Plan& p = *(const Plan*)pv;
  const auto& v = which == 0 ? p.updates : which == 1 ? p.bupdates : p.rupdates;
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].wslot;
}

// The recompute and residual arrays: ritems and yitems as ph_items (8 values
// each), rupdates as ph_updates (7), rsteps {item0, nitems, upd0, nupd, nslots},
// ysteps {item0, nitems}, segsrc.
void ph_rarrays(const void* pv, int64_t* ritems, int32_t* rupd, int32_t* rsteps, int32_t* segsrc, int64_t* yitems,
                int32_t* ysteps) {
  const Plan& p = *(const Plan*)pv;
  auto items = [](const std::vector<scal3r::WorkItem>& v, int64_t* out) {
    for (size_t i = 0; i < v.size(); ++i) {
      const scal3r::WorkItem& w = v[i];
      int64_t* o = out + 8 * i;
      o[0] = w.t0; o[1] = w.t1; o[2] = w.chain; o[3] = w.role;
      o[4] = w.slot; o[5] = w.seq; o[6] = w.wchunk; o[7] = w.aux;
    }
  };
  items(p.ritems, ritems);
  items(p.yitems, yitems);
  for (size_t i = 0; i < p.rupdates.size(); ++i) {
    const scal3r::UpdateItem& u = p.rupdates[i];
    int32_t* o = rupd + 7 * i;
    o[0] = u.chain; o[1] = u.chunk; o[2] = u.slot0; o[3] = u.nslots;
    o[4] = u.last; o[5] = u.seq; o[6] = u.first;
  }
  for (size_t i = 0; i < p.rsteps.size(); ++i) {
    const scal3r::Step& s = p.rsteps[i];
    int32_t* o = rsteps + 5 * i;
    o[0] = s.item0; o[1] = s.nitems; o[2] = s.upd0; o[3] = s.nupd; o[4] = s.nslots;
  }
  for (size_t i = 0; i < p.ysteps.size(); ++i) {
    ysteps[2 * i] = p.ysteps[i].item0;
    ysteps[2 * i + 1] = p.ysteps[i].nitems;
  }
  for (size_t i = 0; i < p.segsrc.size(); ++i) segsrc[i] = p.segsrc[i];
}

}  // extern "C"
