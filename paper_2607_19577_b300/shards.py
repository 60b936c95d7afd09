"""Master-worker evaluation over setting shards, with failure detection.

Sec. III-B partitions the measurement settings among workers: each worker
evaluates its shard (the loss terms, h and G psi restricted to its settings,
normalised by the global B) and the master sums the shard results.  This module
is the host-side coordination of that exchange for ranks that share a
key-value store (torch.distributed's TCPStore; no GPU collective):

* the master splits the settings into shards (replicas.shard) and assigns them
  to the workers it believes alive;
* every worker posts a heartbeat and, per iteration, the result of each shard
  it was assigned;
* a shard whose result does not arrive before the deadline -- its worker died,
  left, or stalls -- is reassigned to a live worker (or evaluated by the master
  itself), and the iteration continues;
* the master adds the shard results in shard order, so the sums do not depend
  on which rank evaluated which shard or on how often a shard was reassigned.

Failures are detected on the host only (missed deadlines, stale heartbeats);
nothing here runs on, or waits inside, a GPU kernel.  A worker leaves only
between shards, never with work of its own in flight."""
from __future__ import annotations

import pickle
import threading
import time
from dataclasses import dataclass, field

from . import replicas

_STOP = "stop"


def _key(*parts) -> str:
    return "/".join(str(p) for p in parts)


@dataclass
class IterationReport:
    """What happened in one master iteration."""
    results: list                       # one result per shard, in shard order
    owner: list                         # rank whose result was used, per shard
    reassigned: dict = field(default_factory=dict)  # shard -> ranks that missed it, in order
    dead: set = field(default_factory=set)          # ranks considered failed after the iteration


class ShardWorker:
    """A worker rank: posts heartbeats and evaluates the shards it is assigned.

    fn(lo, hi) evaluates settings [lo, hi) and returns a picklable result."""

    def __init__(self, store, rank: int, heartbeat_s: float = 0.1):
        self.store, self.rank, self.heartbeat_s = store, rank, heartbeat_s
        self._stop = threading.Event()
        self._hb = threading.Thread(target=self._beat, daemon=True)
        self._hb.start()

    def _beat(self):
        while not self._stop.is_set():
            self.store.set(_key("hb", self.rank), repr(time.time()))
            self._stop.wait(self.heartbeat_s)

    def stop_heartbeat(self):
        """Stop posting heartbeats (a rank that leaves, or a test that plays a dead rank)."""
        self._stop.set()
        self._hb.join()

    def serve(self, fn, poll_s: float = 0.01, max_wait_s: float = 600.0):
        """Answer assignments until the master says stop (or max_wait_s of silence)."""
        seen = 0  # assignment sequence numbers of this rank already served
        idle_since = time.time()
        while True:
            if self.store.check([_STOP]):
                break
            k = _key("assign", self.rank, seen)
            if not self.store.check([k]):
                if time.time() - idle_since > max_wait_s:
                    break
                time.sleep(poll_s)
                continue
            it, shard, lo, hi = pickle.loads(self.store.get(k))
            self.store.set(_key("res", it, shard, self.rank), pickle.dumps(fn(lo, hi)))
            seen += 1
            idle_since = time.time()
        self.store.set(_key("done", self.rank), "1")
        self.stop_heartbeat()


class ShardMaster:
    """The master rank (it also evaluates shards when no worker is left).

    M settings in n_shards contiguous shards (replicas.shard), workers 1..world-1.
    A shard's result is awaited for timeout_s after it was assigned; a worker
    whose heartbeat is older than heartbeat_timeout_s is not assigned work."""

    def __init__(self, store, world: int, M: int, n_shards: int | None = None, timeout_s: float = 1.0,
                 heartbeat_timeout_s: float = 1.0, poll_s: float = 0.005):
        self.store, self.world, self.M = store, world, M
        self.n_shards = n_shards or max(world - 1, 1)
        self.spans = [replicas.shard(M, s, self.n_shards) for s in range(self.n_shards)]
        self.timeout_s, self.hb_timeout_s, self.poll_s = timeout_s, heartbeat_timeout_s, poll_s
        self.dead: set = set()
        self._seq = {r: 0 for r in range(1, world)}  # next assignment number per worker

    def alive(self) -> list:
        """Workers with a fresh heartbeat and no missed deadline."""
        now, out = time.time(), []
        for r in range(1, self.world):
            if r in self.dead:
                continue
            k = _key("hb", r)
            if self.store.check([k]) and now - float(self.store.get(k).decode()) <= self.hb_timeout_s:
                out.append(r)
        return out

    def _assign(self, it, shard, rank):
        lo, hi = self.spans[shard]
        self.store.set(_key("assign", rank, self._seq[rank]), pickle.dumps((it, shard, lo, hi)))
        self._seq[rank] += 1

    def evaluate(self, it: int, fn) -> IterationReport:
        """One iteration: every shard's result, failures handled.  fn(lo, hi) is
        the master's own evaluation, used when no live worker remains."""
        results = [None] * self.n_shards
        owner = [None] * self.n_shards
        reassigned: dict = {}
        pending = {}  # shard -> (rank, deadline)
        live = self.alive()
        for s in range(self.n_shards):
            if live:
                r = live[s % len(live)]
                self._assign(it, s, r)
                pending[s] = (r, time.time() + self.timeout_s)
            else:
                results[s], owner[s] = fn(*self.spans[s]), 0
        while pending:
            for s, (r, deadline) in list(pending.items()):
                k = _key("res", it, s, r)
                if self.store.check([k]):
                    results[s], owner[s] = pickle.loads(self.store.get(k)), r
                    del pending[s]
                elif time.time() > deadline:
                    # missed deadline: the worker is considered failed for good
                    self.dead.add(r)
                    reassigned.setdefault(s, []).append(r)
                    live = self.alive()
                    if live:
                        r2 = live[s % len(live)]
                        self._assign(it, s, r2)
                        pending[s] = (r2, time.time() + self.timeout_s)
                    else:
                        results[s], owner[s] = fn(*self.spans[s]), 0
                        del pending[s]
            time.sleep(self.poll_s)
        return IterationReport(results, owner, reassigned, set(self.dead))

    def stop(self, wait_s: float = 10.0):
        """Tell the workers to stop, then wait (up to wait_s) until each one has
        finished -- the store lives in the master's process -- except workers
        whose heartbeat has gone stale (they have left)."""
        self.store.set(_STOP, "1")
        t0 = time.time()
        for r in range(1, self.world):
            while time.time() - t0 < wait_s and not self.store.check([_key("done", r)]):
                k = _key("hb", r)
                if not self.store.check([k]) or time.time() - float(self.store.get(k).decode()) > self.hb_timeout_s:
                    break
                time.sleep(self.poll_s)


def sum_results(results):
    """Add shard results in shard order (tuples/lists of numpy arrays or floats)."""
    total = None
    for r in results:
        if total is None:
            total = [x.copy() if hasattr(x, "copy") else x for x in r]
        else:
            total = [a + b for a, b in zip(total, r)]
    return total
