"""Minimal best-first branch and bound over node relaxations (Sec. 5.3), the
driver that produces (parent, child) node solves for the learned warm start
and measures it against the parent warm start.

* Node: fixings (int8 p: -1 J0, 0 free, +1 J1), its certified lower bound
  (relax_solve's dual bound) and its solution beta.
* Selection: the open node with the smallest bound.
* Branching: the free coordinate with the largest |beta_j|; children fix it to
  J0 and, while |J1| < k, to J1.
* Incumbent: the support of the k largest |beta_j| (J1 first), solved as the
  node that puts every other coordinate in J0; with no free coordinate the
  relaxation is the restricted problem itself (Eq. 1 on that support), so its
  value is a feasible objective.  Each support is solved once (a cache keyed
  by the support); the batched driver solves a batch's new supports in one
  relax_solve_batch call.
* Pruning: bound >= incumbent - rel_tol * max(1, |incumbent|).
* Warm start of a child: the parent's beta ("parent"), or the learned start
  b + f(x) of include/warmstart.h ("learned"), which falls back to the parent's
  when its certified primal value is not lower.
* Dynamic termination (Sec. 5.3, early-termination rules 1-2), on by default:
  each child is solved with the incumbent's objective as the handle's cutoff
  (relax_set_cutoff), so its loop stops once Phi falls to it (the child will
  be branched) or Psi reaches it (the child is pruned).  Incumbent solves run
  without a cutoff, since they need the restricted optimum.
* Certification: the run is certified only when the queue empties with no
  subtree dropped.  A child left unsolved (max_nodes reached) or whose solve
  failed keeps its parent's bound as the bound of its unexplored subtree, and
  best_bound is the least bound over the queue and those subtrees.

Every relaxation, pass and network evaluation runs in the CUDA library; this
module keeps the queue.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass(order=True)
class Node:
    bound: float
    seq: int
    fix: np.ndarray = field(compare=False)
    beta: object = field(compare=False)       # device tensor (handle dtype)
    iters: int = field(compare=False, default=0)


@dataclass
class BnBStats:
    nodes: int = 0               # node relaxations solved (root and children)
    iters: int = 0               # FISTA iterations of those solves
    incumbent_solves: int = 0    # restricted solves of the incumbent heuristic (not in nodes / iters)
    learned_used: int = 0        # children that started from the network
    fallbacks: int = 0           # children where the parent start was kept
    incumbent: float = float("inf")
    best_bound: float = float("-inf")
    certified: bool = False      # queue emptied and nothing dropped: the incumbent is optimal
    dropped: list = field(default_factory=list)   # parent bounds of children left unsolved or failed
    cut_branch: int = 0          # children stopped by rule 1 (Phi <= incumbent)
    cut_prune: int = 0           # children stopped by rule 2 (Psi >= incumbent)
    seconds: float = 0.0
    pairs: list = field(default_factory=list)   # (parent beta, child fix, child beta) when recording
    bounds: list = field(default_factory=list)  # (parent bound, child's certified bound, cutoff rule) per child


def _branch_var(beta, fix):
    score = np.where(fix == 0, np.abs(beta), -1.0)
    j = int(np.argmax(score))
    return j if score[j] > 0 else -1


def _incumbent_fix(beta, fix, k):
    order = np.argsort(-np.abs(beta), kind="stable")
    sup = list(np.flatnonzero(fix > 0))
    for j in order:
        if len(sup) >= k:
            break
        if fix[j] == 0 and beta[j] != 0:
            sup.append(int(j))
    f = np.full(len(beta), -1, dtype=np.int8)
    f[sup] = 1
    return f


def _finish(st, heap, t0):
    st.certified = not heap and not st.dropped
    st.best_bound = min([n.bound for n in heap] + list(st.dropped), default=st.incumbent)
    st.best_bound = min(st.best_bound, st.incumbent)
    st.seconds = time.perf_counter() - t0
    return st


def run(h, k, max_nodes=50, gap_tol=1e-6, warm="parent", net=None, record=False, rel_tol=1e-9, batch=1,
        cutoff=True):
    """Best-first BnB on the handle's problem; stops when the queue empties
    (certified, unless a subtree was dropped) or after max_nodes relaxations.
    batch > 1: up to `batch` open nodes are taken in best-first order and all
    their children are solved in one relax_solve_batch call (each
    warm-started like a single child).  cutoff: solve children with the
    dynamic termination of Sec. 5.3 against the incumbent."""
    import torch
    dev = h.X.device
    st = BnBStats()
    t0 = time.perf_counter()

    def set_cut(node):
        h.set_cutoff(st.incumbent if (cutoff and node) else float("inf"))

    def count_cut(res):
        st.cut_branch += res.cutoff_rule == 1
        st.cut_prune += res.cutoff_rule == 2

    def solve(fix, start, node=True):
        fx = torch.tensor(fix, device=dev)
        set_cut(node)
        beta, res, code = h.solve(fixings=fx, warm_start=start, gap_tol=gap_tol)
        if node:
            st.nodes += 1
            st.iters += res.iters
            count_cut(res)
        else:
            st.incumbent_solves += 1
        return beta, res, code

    def learned(parent_beta, fix):
        start, used = learned_start(h, net, parent_beta, torch.tensor(fix, device=dev))
        if used:
            st.learned_used += 1
        else:
            st.fallbacks += 1
        return start

    seen = {}   # support -> its restricted objective (inf: solve failed)

    def try_incumbent(beta_np, fix):
        f = _incumbent_fix(beta_np, fix, k)
        key = np.flatnonzero(f > 0).tobytes()
        if key not in seen:
            _, res, code = solve(f, None, node=False)
            seen[key] = res.primal if code in (0, 4) else float("inf")
        if seen[key] < st.incumbent:
            st.incumbent = seen[key]

    def try_incumbents(cands):
        """The incumbent heuristic on several (beta, fix) at once: the new
        supports in one batched solve."""
        new, fixes = [], []
        for beta_np, fix in cands:
            f = _incumbent_fix(beta_np, fix, k)
            key = np.flatnonzero(f > 0).tobytes()
            if key not in seen and key not in new:
                new.append(key)
                fixes.append(f)
        if fixes:
            set_cut(False)
            fixd = torch.tensor(np.stack(fixes), device=dev)
            _, res, _ = h.solve_batch(len(fixes), fixings=fixd, gap_tol=gap_tol)
            st.incumbent_solves += len(fixes)
            for key, r in zip(new, res):
                seen[key] = r.primal if r.status in (0, 4) else float("inf")
        for beta_np, fix in cands:
            key = np.flatnonzero(_incumbent_fix(beta_np, fix, k) > 0).tobytes()
            st.incumbent = min(st.incumbent, seen[key])

    root = np.zeros(h.p, dtype=np.int8)
    beta, res, code = solve(root, None)
    heap = [Node(res.dual_bound, 0, root, beta, res.iters)]
    try_incumbent(beta.double().cpu().numpy(), root)
    seq = 1
    if batch > 1:
        _run_batched(h, k, max_nodes, gap_tol, warm, net, record, rel_tol, batch, heap, st, learned,
                     try_incumbents, dev, set_cut, count_cut)
        h.set_cutoff(float("inf"))
        return _finish(st, heap, t0)
    while heap and st.nodes < max_nodes:
        node = heapq.heappop(heap)
        tol = rel_tol * max(1.0, abs(st.incumbent))
        if node.bound >= st.incumbent - tol:
            continue
        b_np = node.beta.double().cpu().numpy()
        j = _branch_var(b_np, node.fix)
        if j < 0:
            continue
        kids = []
        f0 = node.fix.copy()
        f0[j] = -1
        kids.append(f0)
        if int(np.sum(node.fix > 0)) < k:
            f1 = node.fix.copy()
            f1[j] = 1
            kids.append(f1)
        for f in kids:
            if st.nodes >= max_nodes:
                st.dropped.append(node.bound)      # the sibling's subtree stays unexplored
                break
            start = learned(node.beta, f) if warm == "learned" else node.beta
            beta, res, code = solve(f, start)
            st.bounds.append((node.bound, res.dual_bound, res.cutoff_rule))
            if record:
                st.pairs.append((node.beta.clone(), f.copy(), beta.clone()))
            if code not in (0, 4):
                st.dropped.append(node.bound)      # a failed solve proves nothing about the child
                continue
            # the parent's bound holds for the child too (its feasible set is a
            # subset); a child stopped early by rule 1 may have certified less
            bound = max(res.dual_bound, node.bound)
            if bound < st.incumbent - rel_tol * max(1.0, abs(st.incumbent)):
                heapq.heappush(heap, Node(bound, seq, f, beta, res.iters))
                seq += 1
                try_incumbent(beta.double().cpu().numpy(), f)
    h.set_cutoff(float("inf"))
    return _finish(st, heap, t0)


def _children(node, k):
    """The fixings of a node's children: its branching coordinate to J0 and,
    while |J1| < k, to J1 (none when no free coordinate is nonzero)."""
    j = _branch_var(node.beta.double().cpu().numpy(), node.fix)
    if j < 0:
        return []
    f0 = node.fix.copy()
    f0[j] = -1
    kids = [f0]
    if int(np.sum(node.fix > 0)) < k:
        f1 = node.fix.copy()
        f1[j] = 1
        kids.append(f1)
    return kids


def _run_batched(h, k, max_nodes, gap_tol, warm, net, record, rel_tol, batch, heap, st, learned, try_incumbents,
                 dev, set_cut, count_cut):
    import torch
    seq = 1 << 30
    while heap and st.nodes < max_nodes:
        parents, kids = [], []
        while heap and len(parents) < batch:
            node = heapq.heappop(heap)
            if node.bound >= st.incumbent - rel_tol * max(1.0, abs(st.incumbent)):
                continue
            for f in _children(node, k):
                parents.append(node)
                kids.append(f)
        room = max_nodes - st.nodes
        if not kids:
            continue
        # children beyond the node budget stay unexplored: their parents'
        # bounds remain bounds of those subtrees
        st.dropped.extend(p.bound for p in parents[room:])
        parents, kids = parents[:room], kids[:room]
        fixd = torch.tensor(np.stack(kids), device=dev)
        if warm == "learned":
            warmd, used = learned_starts(h, net, [p.beta for p in parents], fixd)
            st.learned_used += int(used.sum())
            st.fallbacks += int((~used).sum())
        else:
            warmd = torch.stack([p.beta.to(h.dtype) for p in parents]).contiguous()
        set_cut(True)
        betas, res, code = h.solve_batch(len(kids), fixings=fixd, warm_start=warmd, gap_tol=gap_tol)
        pushed = []
        for i, (p, f) in enumerate(zip(parents, kids)):
            r = res[i]
            st.nodes += 1
            st.iters += r.iters + r.polish_iters
            count_cut(r)
            b = betas[i].clone()
            st.bounds.append((p.bound, r.dual_bound, r.cutoff_rule))
            if record:
                st.pairs.append((p.beta.clone(), f.copy(), b))
            if r.status not in (0, 4):
                st.dropped.append(p.bound)
                continue
            bound = max(r.dual_bound, p.bound)
            if bound < st.incumbent - rel_tol * max(1.0, abs(st.incumbent)):
                heapq.heappush(heap, Node(bound, seq, f, b, r.iters))
                seq += 1
                pushed.append((b, f))
        if pushed:
            bs = torch.stack([b.double() for b, _ in pushed]).cpu().numpy()
            try_incumbents([(bs[i], f) for i, (_, f) in enumerate(pushed)])


def learned_start(h, net, parent_beta, fixings):
    """The learned start of a child (fixings: device int8), or the parent's
    beta where the learned start has the higher certified Phi (FP64, +inf
    outside dom g) than the parent's solution on the child's set.  Returns
    (start, used_learned)."""
    feat = h.mlp_features(parent_beta, fixings)
    start = net.predict(feat).to(parent_beta.dtype)
    phi_l, _ = h.certify(start, fixings=fixings)
    phi_p, _ = h.certify(feat[:, 0].contiguous().to(parent_beta.dtype), fixings=fixings)
    if not (phi_l > phi_p):
        return start, True
    return parent_beta, False


def learned_starts(h, net, parent_betas, fixd):
    """learned_start for the children of a batch (fixd: (nb, p) device int8):
    the features of every child, one network evaluation, and the fallback
    test of all 2 nb starts in one relax_certify_batch call.  Returns the
    (nb, p) starts and a boolean numpy mask of the children that kept the
    learned start."""
    import torch
    nb = len(parent_betas)
    feats = torch.cat([h.mlp_features(pb, fixd[i]) for i, pb in enumerate(parent_betas)])
    pred = net.predict(feats).view(nb, h.p).to(h.dtype)
    base = feats[:, 0].contiguous().view(nb, h.p).to(h.dtype)
    vals = h.certify_batch(torch.cat([pred, base]).contiguous(), torch.cat([fixd, fixd]).contiguous())
    used = ~(vals[:nb, 0] > vals[nb:, 0])       # the learned Phi is not higher
    parents = torch.stack([pb.to(h.dtype) for pb in parent_betas])
    mask = torch.tensor(used, device=pred.device)[:, None]
    return torch.where(mask, pred, parents).contiguous(), used


def training_rows(h, pairs):
    """Features, targets of every recorded (parent, child) pair, stacked:
    (rows, 5) float32 and (rows,) float32 device tensors."""
    import torch
    feats, targets = [], []
    for pb, fix, cb in pairs:
        fx = torch.tensor(fix, device=h.X.device)
        feats.append(h.mlp_features(pb, fx).clone())
        targets.append(cb.float())
    return torch.cat(feats), torch.cat(targets)
