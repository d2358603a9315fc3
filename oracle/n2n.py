"""Table 1 as neighbour-to-neighbour message passing, one thread per subgraph — FP64 oracle.
TEST INFRASTRUCTURE ONLY.

The paper runs Table 1 on a distributed computer: every subgraph j repeats steps 3-5 on its own
processor; at iteration k it waits until it has received the pair (u, omega) of iteration k - 1 from
the twin end of each of its lines (step 3, "wait until receiving"), solves eq. 5.8, updates its own
ends and sends each end's new pair to the processor of the twin (step 5).  The library replaces the
messages by a read of the previous sweep's wave buffer on one GPU; this module keeps the messages,
so that their semantics and their failures can be exercised on the host:

* messages carry the iteration number and the sending end, so they may arrive late or out of
  order and the iterates are still exactly those of the synchronous iteration (vtm.VTM.sweep, which
  performs the same arithmetic through VTM.piece_step);
* "wait until receiving" has a time limit: a message that never arrives (dropped) makes the
  waiting subgraph raise N2NTimeout instead of hanging, and every other thread stops at its next
  wait; run() reports the first failure.

Fault injection: ``drop`` is a set of (iteration, end) messages that are never sent; ``delay`` maps
(iteration, end) to seconds the sender sleeps before sending; ``reverse`` sends each subgraph's
messages of an iteration in reverse order.
"""
from __future__ import annotations

import queue
import threading
import time

import numpy as np

from .evs import SplitGraph
from .vtm import VTM, State


class N2NTimeout(RuntimeError):
    """A subgraph waited longer than the limit for a twin's message."""


class N2N:
    def __init__(self, split: SplitGraph, Z, timeout: float = 2.0, drop=(), delay=None, reverse: bool = False):
        self.vtm = VTM(split, Z)
        self.timeout = timeout
        self.drop = set(drop)
        self.delay = dict(delay or {})
        self.reverse = reverse

    def run(self, b: np.ndarray, iterations: int) -> State:
        """Run ``iterations`` iterations of Table 1 from zero boundary variables."""
        m = self.vtm
        b = np.atleast_2d(b)
        R = b.shape[0]
        E = len(m.ends.piece)
        npc = len(m.split.subgraphs)
        inbox = [queue.Queue() for _ in range(npc)]
        stop = threading.Event()
        errors = []
        final_u = np.zeros((R, E))
        final_om = np.zeros((R, E))
        x_local = [None] * npc

        def worker(j: int):
            mine = m.ends_at[j]
            twins = m.ends.twin[mine]
            u = np.zeros((R, E))                 # twins' pair of the previous iteration (step 2: zero)
            om = np.zeros((R, E))
            pending = {}                         # (iteration, end) -> (u, omega), arrived early
            try:
                for k in range(1, iterations + 1):
                    if k > 1:                    # step 3: wait until every twin's pair of k - 1 is here
                        need = {(k - 1, int(t)) for t in twins}
                        while need:
                            have = need & pending.keys()
                            for key in have:
                                tu, to = pending.pop(key)
                                u[:, key[1]] = tu
                                om[:, key[1]] = to
                            need -= have
                            if not need:
                                break
                            if stop.is_set():
                                return
                            try:
                                it, end, tu, to = inbox[j].get(timeout=self.timeout)
                            except queue.Empty:
                                raise N2NTimeout(f"subgraph {j} waited {self.timeout} s for iteration {k - 1}")
                            pending[(it, end)] = (tu, to)
                    new_u = np.zeros((R, E))
                    new_om = np.zeros((R, E))
                    x = m.piece_step(j, u, om, b, new_u, new_om)
                    order = mine[::-1] if self.reverse else mine
                    for t in order:              # step 5: send each end's pair to its twin's subgraph
                        key = (k, int(t))
                        if key in self.drop:
                            continue
                        if key in self.delay:
                            time.sleep(self.delay[key])
                        tw = int(m.ends.twin[t])     # the message is keyed by the sending end
                        inbox[int(m.ends.piece[tw])].put((k, int(t), new_u[:, t].copy(), new_om[:, t].copy()))
                    if k == iterations:
                        final_u[:, mine] = new_u[:, mine]
                        final_om[:, mine] = new_om[:, mine]
                        x_local[j] = x
            except Exception as exc:             # report and stop the others at their next wait
                errors.append(exc)
                stop.set()

        threads = [threading.Thread(target=worker, args=(j,), daemon=True) for j in range(npc)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        if errors:
            raise errors[0]
        return State(u=final_u, omega=final_om, x_local=x_local)
