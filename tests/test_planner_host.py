"""The host-side chunk-step planner, checked without a GPU.

The planner (csrc/plan.cpp) turns a ragged batch into the steps the kernels
run: at forward step j every chain (sequence, head) computes the gradient of
its chunk j at W_j (Eq. 8) and applies W_j to chunk j-1's queries (Eq. 4);
the backward runs the same steps in reverse with the VJPs of both.  Each
task's tokens are cut into 128-token-aligned pieces, and every piece that
feeds an update owns a partial-sum slot.  The tests compile the planner with
g++ and a small C harness (tests/planner_harness.cpp) and check, on ragged
layouts, that

  * every chunk's tokens are covered exactly once per role, in the step the
    recurrence puts them, with boundaries on 128-token tiles;
  * both backward roles of step j read W_j (the checkpoint after chunk j-1,
    or w0 at j = 0);
  * the update items and their slot ranges match the pieces that reduce into
    them;
  * a step never launches more pieces than CTAs (unless it has more tasks),
    and the piece counts minimise the costliest piece (checked against a
    brute-force search);
  * the workspace regions are aligned, disjoint and large enough;
  * malformed layouts are rejected.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import ttt_synth as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_08542_gb300", "csrc")
ALIGN = 128
KEY, APPLY, BKEY, BAPPLY = 0, 1, 2, 3
ERR_INVALID_ARG = 1


def _cuda_include():
    cands = []
    nvcc = shutil.which("nvcc")
    if nvcc:
        cands.append(os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include"))
    cands += ["/usr/local/cuda/include"]
    for c in cands:
        if os.path.exists(os.path.join(c, "cuda_runtime.h")):
            return c
    return None


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("planner") / "libplanner_harness.so")
    cmd = [cxx, "-std=c++17", "-O1", "-fPIC", "-shared", "-I" + inc, "-I" + os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "planner_harness.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(out)
    P = ctypes.POINTER
    L.ph_build_opts.restype = ctypes.c_void_p
    L.ph_build_opts.argtypes = [ctypes.c_int32] * 4 + [P(ctypes.c_int32), P(ctypes.c_float), P(ctypes.c_int64),
                                                       ctypes.c_int32, P(ctypes.c_int32), ctypes.c_int32,
                                                       ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32)]
    L.ph_counts2.argtypes = [ctypes.c_void_p, P(ctypes.c_int64)]
    L.ph_bsteps2.argtypes = [ctypes.c_void_p, P(ctypes.c_int32)]
    L.ph_nfill.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int32)]
    L.ph_wslots.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int32)]
    L.ph_rarrays.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_int32),
                             P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_int32)]
    L.ph_free.argtypes = [ctypes.c_void_p]
    L.ph_counts.argtypes = [ctypes.c_void_p, P(ctypes.c_int64)]
    L.ph_items.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int64)]
    L.ph_updates.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int32)]
    L.ph_steps.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int32)]
    L.ph_workspace.restype = ctypes.c_int64
    L.ph_workspace.argtypes = [ctypes.c_void_p] + [ctypes.c_int32] * 4
    L.ph_carve.argtypes = [ctypes.c_void_p] + [ctypes.c_int32] * 4 + [ctypes.c_int64, P(ctypes.c_int64)]
    L.ph_bwd_scratch_tiles_per_piece.restype = ctypes.c_int32
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class PlanView:
    """The plan read back into numpy arrays."""

    def __init__(self, lib, H, off, ptr, num_sms=152, ctas=0, fwd_waves=1, bwd_waves=1, min_tokens=256,
                 key_cost=1.85, bkey_cost=2.25, D=64, F=128, align=ALIGN, ckpt_every=1, mse_compose=False,
                 fill=0):
        self.lib, self.H, self.D, self.F = lib, H, D, F
        self.align, self.ckpt_every, self.mse_compose = align, ckpt_every, mse_compose
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.ptr = np.ascontiguousarray(ptr, dtype=np.int32)
        self.sched = dict(num_sms=num_sms, ctas=ctas, fwd_waves=fwd_waves, bwd_waves=bwd_waves,
                          min_tokens=min_tokens, key_cost=np.float32(key_cost), bkey_cost=np.float32(bkey_cost),
                          fill=fill)
        sch = np.array([ctas, fwd_waves, bwd_waves, min_tokens, align, fill], dtype=np.int32)
        costs = np.array([key_cost, bkey_cost], dtype=np.float32)
        rc = ctypes.c_int32(-1)
        self.h = lib.ph_build_opts(H, D, F, num_sms, _ptr(sch, ctypes.c_int32), _ptr(costs, ctypes.c_float),
                                   _ptr(self.off, ctypes.c_int64), len(self.off) - 1,
                                   _ptr(self.ptr, ctypes.c_int32), len(self.ptr) - 1, ckpt_every,
                                   int(mse_compose), ctypes.byref(rc))
        self.rc = rc.value
        if not self.h:
            return
        cnt = np.zeros(10, dtype=np.int64)
        lib.ph_counts(self.h, _ptr(cnt, ctypes.c_int64))
        (n_it, n_up, n_st, self.max_slots, n_bit, n_bup, n_bst, self.bmax_slots, self.bscratch,
         self.max_chunks) = (int(x) for x in cnt)
        self.items, self.updates, self.steps = self._read(0, n_it, n_up, n_st)
        self.bitems, self.bupdates, self.bsteps = self._read(1, n_bit, n_bup, n_bst)
        c2 = np.zeros(8, dtype=np.int64)
        lib.ph_counts2(self.h, _ptr(c2, ctypes.c_int64))
        n_ri, n_ru, n_rs, n_seg, n_yi, n_ys, self.ckpt_slots, _ = (int(x) for x in c2)
        self.bsteps2 = np.zeros((max(n_bst, 1), 5), dtype=np.int32)
        if n_bst:
            lib.ph_bsteps2(self.h, _ptr(self.bsteps2, ctypes.c_int32))
        self.bsteps2 = self.bsteps2[:n_bst]
        # tail-fill pieces at the end of every step (forward, backward)
        self.nfill = []
        for bwd, n in ((0, n_st), (1, n_bst)):
            nf = np.zeros(max(n, 1), dtype=np.int32)
            if n:
                lib.ph_nfill(self.h, bwd, _ptr(nf, ctypes.c_int32))
            self.nfill.append(nf[:n])
        self.wslots = []
        for which, n in ((0, n_up), (1, n_bup), (2, n_ru)):
            w = np.zeros(max(n, 1), dtype=np.int32)
            if n:
                lib.ph_wslots(self.h, which, _ptr(w, ctypes.c_int32))
            self.wslots.append(w[:n])
        self.ritems = np.zeros((max(n_ri, 1), 8), dtype=np.int64)
        self.rupdates = np.zeros((max(n_ru, 1), 7), dtype=np.int32)
        self.rsteps = np.zeros((max(n_rs, 1), 5), dtype=np.int32)
        self.segsrc = np.zeros(max(n_seg, 1), dtype=np.int32)
        self.yitems = np.zeros((max(n_yi, 1), 8), dtype=np.int64)
        self.ysteps = np.zeros((max(n_ys, 1), 2), dtype=np.int32)
        lib.ph_rarrays(self.h, _ptr(self.ritems, ctypes.c_int64), _ptr(self.rupdates, ctypes.c_int32),
                       _ptr(self.rsteps, ctypes.c_int32), _ptr(self.segsrc, ctypes.c_int32),
                       _ptr(self.yitems, ctypes.c_int64), _ptr(self.ysteps, ctypes.c_int32))
        self.ritems, self.rupdates, self.rsteps = self.ritems[:n_ri], self.rupdates[:n_ru], self.rsteps[:n_rs]
        self.segsrc, self.yitems, self.ysteps = self.segsrc[:n_seg], self.yitems[:n_yi], self.ysteps[:n_ys]

    def _read(self, bwd, n_it, n_up, n_st):
        it = np.zeros((n_it, 8), dtype=np.int64)
        up = np.zeros((n_up, 7), dtype=np.int32)
        st = np.zeros((n_st, 6), dtype=np.int32)
        if n_it:
            self.lib.ph_items(self.h, bwd, _ptr(it, ctypes.c_int64))
        if n_up:
            self.lib.ph_updates(self.h, bwd, _ptr(up, ctypes.c_int32))
        if n_st:
            self.lib.ph_steps(self.h, bwd, _ptr(st, ctypes.c_int32))
        return it, up, st

    def close(self):
        if self.h:
            self.lib.ph_free(self.h)
            self.h = None

    # ---- helpers -------------------------------------------------------
    @property
    def S(self):
        return len(self.ptr) - 1

    def nchunks(self, q):
        return int(self.ptr[q + 1] - self.ptr[q])

    def chunk_of(self, t0, t1):
        c = int(np.searchsorted(self.off, t0, side="right")) - 1
        assert 0 <= c < len(self.off) - 1 and self.off[c] <= t0 < t1 <= self.off[c + 1], (t0, t1)
        return c

    def step_items(self, bwd, s):
        st = (self.bsteps if bwd else self.steps)[s]
        return (self.bitems if bwd else self.items)[st[0]:st[0] + st[1]]

    def step_updates(self, bwd, s):
        st = (self.bsteps if bwd else self.steps)[s]
        return (self.bupdates if bwd else self.updates)[st[2]:st[2] + st[3]]

    def ctas(self, bwd):
        c = self.sched["ctas"] or self.sched["num_sms"]
        return c * (self.sched["bwd_waves"] if bwd else self.sched["fwd_waves"])

    def cost(self, role, length):
        if role == KEY:
            return length * float(self.sched["key_cost"])
        if role == BKEY:
            return length * float(self.sched["bkey_cost"])
        return float(length)


def _expected_tasks(pv, bwd, s):
    """(chain, role, chunk, wchunk) of every task at step s, from the recurrence."""
    maxn = pv.max_chunks
    j = maxn - s if bwd else s
    out = []
    for q in range(pv.S):
        n = pv.nchunks(q)
        for h in range(pv.H):
            chain = q * pv.H + h
            if not bwd:
                if j < n:
                    out.append((chain, KEY, int(pv.ptr[q]) + j, -1))
                if 1 <= j <= n:
                    out.append((chain, APPLY, int(pv.ptr[q]) + j - 1, -1))
            elif n >= 1 and j <= n:
                w = int(pv.ptr[q]) + j - 1 if j >= 1 else -1   # checkpoint holding W_j
                if j < n:
                    out.append((chain, BKEY, int(pv.ptr[q]) + j, w))
                if j >= 1:
                    out.append((chain, BAPPLY, int(pv.ptr[q]) + j - 1, w))
    return out


def _group_pieces(pv, items):
    """pieces grouped by task (chain, role, chunk) -> list of item rows."""
    g = {}
    for r in items:
        c = pv.chunk_of(int(r[0]), int(r[1]))
        g.setdefault((int(r[2]), int(r[3]), c), []).append(r)
    return g


def _check_plan(pv):
    assert pv.rc == 0 and pv.h
    maxn = max((pv.nchunks(q) for q in range(pv.S)), default=0)
    assert pv.max_chunks == maxn
    assert len(pv.steps) == maxn + 1 and len(pv.bsteps) == maxn + 1
    seen = {}
    per_piece_tiles = pv.lib.ph_bwd_scratch_tiles_per_piece()
    max_scratch = 0
    for bwd in (0, 1):
        steps = pv.bsteps if bwd else pv.steps
        # the steps' item and update ranges tile the plan's arrays in order
        assert np.array_equal(steps[:, 0], np.concatenate([[0], np.cumsum(steps[:, 1])[:-1]]))
        assert np.array_equal(steps[:, 2], np.concatenate([[0], np.cumsum(steps[:, 3])[:-1]]))
        assert steps[:, 1].sum() == len(pv.bitems if bwd else pv.items)
        for s in range(len(steps)):
            items = pv.step_items(bwd, s)
            ups = pv.step_updates(bwd, s)
            want = _expected_tasks(pv, bwd, s)
            groups = _group_pieces(pv, items)
            assert sorted(groups) == sorted((c, r, k) for c, r, k, _ in want), (bwd, s)
            wchunk = {(c, r, k): w for c, r, k, w in want}
            for (chain, role, c), pcs in groups.items():
                pcs = sorted(pcs, key=lambda r: r[0])
                t0, t1 = int(pv.off[c]), int(pv.off[c + 1])
                # exact cover of the chunk, 128-token boundaries from its start
                assert pcs[0][0] == t0 and pcs[-1][1] == t1
                for a, b in zip(pcs[:-1], pcs[1:]):
                    assert a[1] == b[0]
                for r in pcs:
                    assert r[1] > r[0] and (r[0] - t0) % pv.align == 0
                    assert r[5] == chain // pv.H
                    if bwd:
                        assert r[6] == wchunk[(chain, role, c)]
                key = (bwd, role, chain, c)
                assert key not in seen
                seen[key] = len(pcs)
            # the costliest pieces come first (the first wave; tail-fill pieces
            # follow it)
            nf = int(pv.nfill[bwd][s])
            first = items[:len(items) - nf]
            costs = [pv.cost(int(r[3]), int(r[1] - r[0])) for r in first]
            assert all(costs[i] >= costs[i + 1] * (1 - 1e-6) for i in range(len(costs) - 1))
            # no more pieces than CTAs, unless the step has more tasks than
            # CTAs; the fill adds at most one more wave
            assert len(first) <= max(len(want), pv.ctas(bwd))
            assert nf == 0 or (pv.sched["fill"] & (2 if bwd else 1) and nf <= pv.ctas(bwd))
            # updates: one per chain that closes a chunk here, in sequence-major order
            _check_updates(pv, bwd, s, items, ups)
            st = steps[s]
            assert st[4] == sum(int(u[3]) for u in ups)
            if bwd:
                tiles = 0
                for r in items:
                    assert r[7] == tiles
                    if r[3] == BKEY:
                        tiles += per_piece_tiles
                assert st[5] == tiles
                max_scratch = max(max_scratch, tiles)
            else:
                assert (items[:, 7] == 0).all()
        assert (pv.bmax_slots if bwd else pv.max_slots) == max(int(st[4]) for st in steps)
    assert pv.bscratch == max_scratch
    # every chunk of every chain appears once per role over the whole plan
    for q in range(pv.S):
        for c in range(int(pv.ptr[q]), int(pv.ptr[q + 1])):
            for h in range(pv.H):
                for bwd, role in ((0, KEY), (0, APPLY), (1, BKEY), (1, BAPPLY)):
                    assert (bwd, role, q * pv.H + h, c) in seen


def _check_updates(pv, bwd, s, items, ups):
    j = pv.max_chunks - s if bwd else s
    want = []
    for q in range(pv.S):
        n = pv.nchunks(q)
        for h in range(pv.H):
            chain = q * pv.H + h
            if not bwd:
                if j < n:
                    want.append((chain, int(pv.ptr[q]) + j, int(j == n - 1), q, 0))
                elif n == 0 and j == 0:
                    want.append((chain, -1, 1, q, 0))   # empty sequence: w_final = w0
            elif n >= 1 and j <= n:
                want.append((chain, int(pv.ptr[q]) + j - 1 if j >= 1 else -1, int(j == n), q, int(j == 0)))
    got = [(int(u[0]), int(u[1]), int(u[4]), int(u[5]), int(u[6]) if bwd else 0) for u in ups]
    assert got == want, (bwd, s)
    # slots: each update owns a contiguous range holding exactly the slots of
    # the pieces of its chain that reduce (key pieces forward, all backward)
    slot = 0
    for u in ups:
        assert u[2] == slot
        mine = sorted(int(r[4]) for r in items if r[2] == u[0] and (bwd or r[3] == KEY))
        assert mine == list(range(int(u[2]), int(u[2] + u[3])))
        slot += int(u[3])
    if not bwd:
        assert (items[items[:, 3] == APPLY][:, 4] == -1).all()
    assert (items[:, 4] < slot).all()


def _optimal_max_cost(costs, caps, ctas):
    """Smallest achievable max_i cost_i / m_i with 1 <= m_i <= caps_i and
    sum m_i <= max(ctas, ntasks), by trying every candidate value."""
    budget = max(ctas, len(costs))
    best = math.inf
    cands = sorted({c / m for c, cap in zip(costs, caps) for m in range(1, cap + 1)})
    for x in cands:
        need = 0
        ok = True
        for c, cap in zip(costs, caps):
            m = max(1, math.ceil(c / x - 1e-9))
            if m > cap:
                ok = False
                break
            need += m
        if ok and need <= budget:
            best = min(best, x)
    return best


def _check_minmax(pv):
    """The piece counts minimise the costliest piece of every step (the
    first wave's counts, when the tail fill adds pieces behind it)."""
    mt = pv.sched["min_tokens"]
    for bwd in (0, 1):
        steps = pv.bsteps if bwd else pv.steps
        for s in range(len(steps)):
            items = pv.step_items(bwd, s)
            groups = _group_pieces(pv, items[:len(items) - int(pv.nfill[bwd][s])])
            costs, caps, got = [], [], 0.0
            for (chain, role, c), pcs in groups.items():
                length = int(pv.off[c + 1] - pv.off[c])
                cost = float(np.float32(pv.cost(role, length)))
                tiles = -(-length // pv.align)
                cap = 1
                while cap + 1 <= tiles and length // (cap + 1) >= mt:
                    cap += 1
                costs.append(cost)
                caps.append(cap)
                assert 1 <= len(pcs) <= cap
                got = max(got, cost / len(pcs))
            if costs:
                want = _optimal_max_cost(costs, caps, pv.ctas(bwd))
                assert got <= want * (1 + 1e-5), (bwd, s, got, want)


LAYOUTS = {
    "one chunk": [[300]],
    "ragged, two seqs": [[300, 129, 77], [513]],
    "tiny chunks": [[1, 2, 127, 128, 129]],
    "empty sequence between": [[1041 * 2, 700], [], [5000, 64, 1]],
    "many short seqs": [[200, 100]] * 7 + [[4096]],
}


@pytest.mark.parametrize("fill", [0, 3])
@pytest.mark.parametrize("name", list(LAYOUTS))
@pytest.mark.parametrize("H,num_sms,ctas,waves,min_tokens", [(1, 152, 0, 1, 256), (4, 8, 0, 2, 128),
                                                            (3, 152, 20, 1, 512), (16, 4, 0, 1, 256)])
def test_plan_invariants_on_ragged_layouts(lib, name, H, num_sms, ctas, waves, min_tokens, fill):
    lay = syn.layout_from_lengths(LAYOUTS[name])
    pv = PlanView(lib, H, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=num_sms, ctas=ctas, fwd_waves=waves,
                  bwd_waves=waves, min_tokens=min_tokens, fill=fill)
    try:
        _check_plan(pv)
        _check_minmax(pv)
    finally:
        pv.close()


@pytest.mark.parametrize("wl,H", [("bf16_vggt64", 16), ("bf16_ragged24", 16), ("bf16_vggt64", 1)])
def test_plan_invariants_on_benchmark_layouts(lib, wl, H):
    """The benchmark's own layouts: 66,624 tokens in 16-frame chunks, and 24
    ragged sequences; 16 heads, or one head (the AMU shape)."""
    lay = syn.workload(wl).layout()
    pv = PlanView(lib, H, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=152)
    try:
        _check_plan(pv)
        _check_minmax(pv)
        if wl == "bf16_vggt64" and H == 16:
            # 16 chains x (key + apply) = 32 tasks; the planner fills the SMs
            full = [len(pv.step_items(0, s)) for s in range(1, len(pv.steps) - 1)]
            assert all(n == 152 for n in full), full
    finally:
        pv.close()


# ---- the tail fill -----------------------------------------------------------
# The planner's piece-time model (units of the step's cheaper token): a fixed
# cost per piece, a cost per token of whole tiles, and for an update-VJP piece
# a cost per sub-piece of four tiles; a CTA behind the first wave starts a
# little after its SM frees.
_FILL_OVH = {KEY: 544.0, APPLY: 427.0, BKEY: 568.0, BAPPLY: 60.0}


def _fill_time(pv, role, length):
    tiles = -(-length // pv.align)
    t = float(tiles * pv.align)
    if role == KEY:
        return _FILL_OVH[KEY] + t * 2.42
    if role == BKEY:
        return _FILL_OVH[BKEY] + t * 2.15 + -(-tiles // 4) * 30.0
    return _FILL_OVH[role] + t


def _dispatch_end(pv, items, ctas, start_lag=32.0):
    """When the last piece of a launch ends if the GPU starts CTA k on the
    first SM that frees once CTAs 0..k-1 have started."""
    import heapq
    free, end = [], 0.0
    for k, r in enumerate(items):
        t = _fill_time(pv, int(r[3]), int(r[1] - r[0]))
        if k < ctas:
            e = t
        else:
            e = heapq.heappop(free) + start_lag + t
        heapq.heappush(free, e)
        end = max(end, e)
    return end


def _task_counts(pv, items):
    return {k: len(v) for k, v in _group_pieces(pv, items).items()}


@pytest.mark.parametrize("wl,H", [("bf16_vggt64", 16), ("bf16_window256", 16), ("bf16_fwdbwd_2x32", 16)])
def test_tail_fill_on_benchmark_layouts(lib, wl, H):
    """The fill leaves each task's first-wave piece count as the one-wave plan
    has it, covers the rest behind the first wave, and shortens every launch it
    touches under the model by at least the planner's 2 % margin, with the GPU's
    dispatch order simulated from the item order alone."""
    lay = syn.workload(wl).layout()
    one = PlanView(lib, H, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=152)
    pv = PlanView(lib, H, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=152, fill=3)
    try:
        _check_plan(pv)
        _check_minmax(pv)
        touched = 0
        for bwd in (0, 1):
            steps = pv.bsteps if bwd else pv.steps
            for s in range(len(steps)):
                a, b = one.step_items(bwd, s), pv.step_items(bwd, s)
                nf = int(pv.nfill[bwd][s])
                assert int(one.nfill[bwd][s]) == 0
                if nf == 0:
                    assert np.array_equal(a, b)
                    continue
                touched += 1
                assert _task_counts(pv, b[:len(b) - nf]) == _task_counts(one, a)
                # fill pieces: whole tiles, or the ragged end of their task
                for r in b[len(b) - nf:]:
                    c = pv.chunk_of(int(r[0]), int(r[1]))
                    assert (r[1] - r[0]) % pv.align == 0 or r[1] == pv.off[c + 1]
                t_one, t_fill = _dispatch_end(one, a, 152), _dispatch_end(pv, b, 152)
                assert t_fill <= 0.98 * t_one + 1e-6, (bwd, s, t_fill, t_one)
        if wl == "bf16_vggt64":
            # the three steps with both roles, in each direction
            assert [int(x) > 0 for x in pv.nfill[0]] == [False, True, True, True, False]
            assert [int(x) > 0 for x in pv.nfill[1]] == [False, True, True, True, False]
        assert touched > 0
    finally:
        pv.close()
        one.close()


def test_tail_fill_off_keeps_the_one_wave_plan(lib):
    """fill = 0 never adds a piece, and neither does fill = 3 with more than
    one wave or when the one-wave plan is already balanced."""
    lay = syn.workload("bf16_vggt64").layout()
    for kw in ({"fill": 0}, {"fill": 3, "fwd_waves": 2, "bwd_waves": 2}):
        pv = PlanView(lib, 16, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=152, **kw)
        try:
            assert all((nf == 0).all() for nf in pv.nfill)
        finally:
            pv.close()
    bal = syn.layout_from_lengths([[256 * 152]])   # every step: one task, 152 pieces of two tiles
    pv = PlanView(lib, 1, bal.chunk_offsets, bal.seq_chunk_ptr, num_sms=152, fill=3)
    try:
        _check_plan(pv)
        assert all((nf == 0).all() for nf in pv.nfill)
    finally:
        pv.close()


def test_pieces_stop_at_the_tile_and_min_token_limits(lib):
    """With CTAs to spare, every task is cut until one more cut would give a
    piece under min_tokens or under one tile."""
    lay = syn.layout_from_lengths([[1000, 257, 128 * 9 + 5]])
    for mt in (1, 128, 300):
        pv = PlanView(lib, 1, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=10_000, min_tokens=mt)
        try:
            _check_plan(pv)
            for bwd in (0, 1):
                steps = pv.bsteps if bwd else pv.steps
                for s in range(len(steps)):
                    for (_, _, c), pcs in _group_pieces(pv, pv.step_items(bwd, s)).items():
                        length = int(pv.off[c + 1] - pv.off[c])
                        m = len(pcs)
                        tiles = -(-length // pv.align)
                        assert m + 1 > tiles or length // (m + 1) < mt, (mt, length, m)
        finally:
            pv.close()


def test_more_tasks_than_ctas_gives_one_piece_each(lib):
    lay = syn.layout_from_lengths([[4096, 4096]] * 3)
    pv = PlanView(lib, 8, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=16)
    try:
        _check_plan(pv)
        for bwd in (0, 1):
            steps = pv.bsteps if bwd else pv.steps
            for s in range(len(steps)):
                groups = _group_pieces(pv, pv.step_items(bwd, s))
                if len(groups) >= 16:
                    assert all(len(p) == 1 for p in groups.values())
    finally:
        pv.close()


def test_all_sequences_empty(lib):
    """No chunks at all: one forward step of updates that copy w0 to
    w_final, and no backward work."""
    pv = PlanView(lib, 2, [0], [0, 0, 0])
    try:
        assert pv.rc == 0
        assert len(pv.items) == 0 and len(pv.bitems) == 0
        assert [tuple(u[:2]) for u in pv.updates] == [(0, -1), (1, -1), (2, -1), (3, -1)]
        assert (pv.updates[:, 3] == 0).all() and (pv.updates[:, 4] == 1).all()
        assert pv.max_slots == 0 and pv.bscratch == 0
    finally:
        pv.close()


@pytest.mark.parametrize("off,ptr", [
    ([1, 100], [0, 1]),             # first offset not 0
    ([0, 100, 100], [0, 2]),        # empty chunk
    ([0, 100, 50], [0, 2]),         # decreasing offsets
    ([0, 100], [1, 1]),             # first pointer not 0
    ([0, 100, 200], [0, 1]),        # pointers do not end at C
    ([0, 100, 200], [0, 2, 1, 2]),  # decreasing pointers
    ([0, 100], [0]),                # no sequence
    ([0, (1 << 40) + 1], [0, 1]),   # more tokens than the planner allows
])
def test_malformed_layouts_rejected(lib, off, ptr):
    pv = PlanView(lib, 2, off, ptr)
    assert pv.rc == ERR_INVALID_ARG and not pv.h


@pytest.mark.parametrize("H,D,F", [(16, 64, 128), (1, 256, 1024), (2, 16, 32)])
def test_workspace_regions_aligned_disjoint_and_sized(lib, H, D, F):
    lay = syn.layout_from_lengths([[2000, 1041, 77], [333], []])
    pv = PlanView(lib, H, lay.chunk_offsets, lay.seq_chunk_ptr, num_sms=32, D=D, F=F)
    try:
        chains = pv.S * H
        P, R = 3 * F * D, 2 * F + D
        total = {b: pv.lib.ph_workspace(pv.h, H, D, F, b) for b in (0, 1)}
        assert total[1] > total[0] > 0
        for bwd in (0, 1):
            base = 1 << 20
            o = np.zeros(7, dtype=np.int64)
            pv.lib.ph_carve(pv.h, H, D, F, bwd, base, _ptr(o, ctypes.c_int64))
            slots = max(pv.max_slots, pv.bmax_slots if bwd else 0, 1)
            sizes = [2 * chains * P * 4, chains * R * 4, slots * P * 4]
            if bwd:
                sizes += [chains * P * 4, chains * R * 4, chains * P * 4, pv.bscratch * 3 * 32 * 1024]
            else:
                assert (o[3:] == -1).all()
            regions = [(int(o[i]), sizes[i]) for i in range(len(sizes))]
            for i, (start, size) in enumerate(regions):
                assert start % (1024 if i == 6 else 256) == 0
                end = start + size
                assert end <= total[bwd]
                if i + 1 < len(regions):
                    assert end <= regions[i + 1][0]
    finally:
        pv.close()


# ---- the float32 path's 16-token pieces ------------------------------------

def test_float32_tiles_split_short_chunks(lib):
    """The float32 kernels work in 16-token tiles, so their plan cuts on 16
    tokens with no larger minimum: with CTAs free, a 128-token chunk becomes
    eight pieces per role (the 8-chunk, 128-token workload)."""
    lay = syn.layout_from_lengths([[128] * 8])
    pv = PlanView(lib, 1, lay.chunk_offsets, lay.seq_chunk_ptr, align=16, min_tokens=16)
    try:
        _check_plan(pv)
        for bwd in (0, 1):
            for s in range(len(pv.bsteps if bwd else pv.steps)):
                for pcs in _group_pieces(pv, pv.step_items(bwd, s)).values():
                    assert len(pcs) == 8 and all(int(r[1] - r[0]) == 16 for r in pcs)
    finally:
        pv.close()


# ---- sparse checkpoints ------------------------------------------------------

SPARSE_LENS = [[300, 129, 77, 200, 50], [130, 257], [100, 100, 100], [64]]


@pytest.mark.parametrize("fill", [0, 3])
@pytest.mark.parametrize("n", [2, 3, 5])
def test_sparse_checkpoint_plan(lib, n, fill):
    """ckpt_every = n: the forward writes the weights after local chunks
    n-1, 2n-1, ... to consecutive slots, sequence after sequence; every
    backward step reads W_j from its slot (j a multiple of n), w0 (j = 0) or
    the recompute buffer at the sequence's row; the first backward step of a
    segment reruns the forward steps that rebuild it, with the forward's own
    pieces and partial slots (tail-fill pieces included)."""
    lay = syn.layout_from_lengths(SPARSE_LENS)
    pv = PlanView(lib, 2, lay.chunk_offsets, lay.seq_chunk_ptr, ckpt_every=n, fill=fill)
    try:
        assert pv.rc == 0
        nch = [len(x) for x in SPARSE_LENS]
        base = np.concatenate([[0], np.cumsum([c // n for c in nch])])
        assert pv.ckpt_slots == base[-1]
        for u, w in zip(pv.updates, pv.wslots[0]):
            chunk, q = int(u[1]), int(u[5])
            if chunk < 0:
                assert w == -1
                continue
            j = chunk - int(pv.ptr[q])
            assert w == (base[q] + (j + 1) // n - 1 if (j + 1) % n == 0 else -1)
        maxn = pv.max_chunks

        def source(q, j):
            return -1 if j == 0 else (q if j % n else base[q] + j // n - 1)

        tops = []
        for s in range(len(pv.bsteps)):
            j = maxn - s
            wseg, rec0, nrec, segk, npost = (int(x) for x in pv.bsteps2[s])
            assert wseg == j % n and npost == 0
            top = j % n != 0 and (j == maxn or (j + 1) % n == 0)
            assert (nrec > 0) == top
            if top:
                assert rec0 == j - j % n and nrec == j % n and segk == j // n
                tops.append(j)
            for r in pv.step_items(1, s):
                assert r[6] == source(int(r[5]), j)
            st = pv.bsteps[s]
            for u, w in zip(pv.bupdates[st[2]:st[2] + st[3]], pv.wslots[1][st[2]:st[2] + st[3]]):
                if j >= 1:
                    assert w == source(int(u[5]), j)
        # every W_j read from the recompute buffer is rebuilt by its segment's first step
        for j in range(1, maxn + 1):
            if j % n:
                assert any(t - t % n == j - j % n and t >= j for t in tops), j
        assert len(pv.rsteps) == maxn
        for j in range(maxn):
            fi = np.array([r for r in pv.step_items(0, j) if r[3] == KEY]).reshape(-1, 8)
            rs = pv.rsteps[j]
            assert np.array_equal(pv.ritems[rs[0]:rs[0] + rs[1]], fi)
            assert rs[4] == pv.steps[j][4]
            fu = [u for u in pv.step_updates(0, j) if u[1] >= 0]
            ru = pv.rupdates[rs[2]:rs[2] + rs[3]]
            assert len(fu) == len(ru)
            for a, b, w in zip(fu, ru, pv.wslots[2][rs[2]:rs[2] + rs[3]]):
                assert tuple(a[:4]) == tuple(b[:4]) and b[4] == 0 and w == b[5]
        nseg = maxn // n + 1
        assert len(pv.segsrc) == nseg * pv.S
        for k in range(nseg):
            for q in range(pv.S):
                want = -2 if k * n > nch[q] else (-1 if k == 0 else base[q] + k - 1)
                assert pv.segsrc[k * pv.S + q] == want
    finally:
        pv.close()


def test_dense_checkpoints_plan_no_recompute(lib):
    lay = syn.layout_from_lengths(SPARSE_LENS)
    pv = PlanView(lib, 2, lay.chunk_offsets, lay.seq_chunk_ptr)
    try:
        _check_plan(pv)
        assert pv.ckpt_slots == len(pv.off) - 1
        assert (pv.bsteps2 == 0).all() and len(pv.rsteps) == 0 and len(pv.segsrc) == 0
        for u, w in zip(pv.updates, pv.wslots[0]):
            assert w == u[1]
    finally:
        pv.close()


# ---- the composed squared-error loss (BF16, head_dim 64) -------------------

@pytest.mark.parametrize("fill", [0, 3])
def test_composed_mse_plan(lib, fill):
    """Forward: each step's residual pieces are its gradient pieces as apply
    pieces.  Backward: the last npost pieces of a step are the key-side apply
    VJPs; they cover the same tokens as the step's update VJPs, read the same
    weights, and reduce into their chain's slots like every other piece.  The
    tail fill stays off: part of each backward step is launched separately,
    outside its one-launch model."""
    lay = syn.layout_from_lengths([[300, 129, 77], [130, 257], [64]])
    H = 2
    pv = PlanView(lib, H, lay.chunk_offsets, lay.seq_chunk_ptr, mse_compose=True, fill=fill)
    try:
        assert pv.rc == 0
        assert all((nf == 0).all() for nf in pv.nfill)
        maxn = pv.max_chunks
        assert len(pv.ysteps) == maxn + 1
        for j in range(maxn + 1):
            fi = [r for r in pv.step_items(0, j) if r[3] == KEY]
            ys = pv.ysteps[j]
            yi = pv.yitems[ys[0]:ys[0] + ys[1]]
            assert len(yi) == len(fi)
            for a, b in zip(fi, yi):
                assert tuple(a[:3]) == tuple(b[:3]) and b[3] == APPLY and b[4] == -1 and b[5] == a[5]

        def cover(rows):
            return {(int(r[2]), t) for r in rows for t in range(int(r[0]), int(r[1]))}

        for s in range(len(pv.bsteps)):
            items = pv.step_items(1, s)
            npost = int(pv.bsteps2[s][4])
            main, post = items[:len(items) - npost], items[len(items) - npost:]
            assert (post[:, 3] == 4).all() and (main[:, 3] != 4).all()
            bkey = main[main[:, 3] == BKEY]
            assert cover(bkey) == cover(post)
            w = {int(r[2]): int(r[6]) for r in bkey}
            assert all(w[int(r[2])] == r[6] for r in post)
            ups = pv.step_updates(1, s)
            rng = {int(u[0]): (int(u[2]), int(u[2]) + int(u[3])) for u in ups}
            for r in items:
                a, b = rng[int(r[2])]
                assert a <= r[4] < b
            assert sorted(int(r[4]) for r in items) == list(range(int(pv.bsteps[s][4])))
    finally:
        pv.close()
