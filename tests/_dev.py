"""Test-side wrapper around the C-ABI binding: moves numpy inputs to the
device with torch and calls the cupc_* entry points. Marshalling only."""
import numpy as np
import torch

from paper_2509_14433_gb300 import cupc as C


class Dev:
    def __init__(self, V, seed, params=None, workspace=None):
        self.V = V
        st, self.h = C.cupc_init(V, seed, params, workspace, None)
        C.check(st, "cupc_init")
        p = np.zeros(4, np.uint32)
        C.check(C.cupc_get_params(self.h, p))
        self.L, self.C, self.D, self.W = (int(x) for x in p)

    def close(self):
        if self.h:
            C.cupc_destroy(self.h)
            self.h = None

    __del__ = close

    def update(self, edges, ops=None, host=False):
        e = np.ascontiguousarray(np.asarray(edges, np.uint32).reshape(-1))
        n = e.size // 2
        o = np.ones(n, np.int8) if ops is None else np.ascontiguousarray(np.asarray(ops, np.int8))
        if host:
            return C.cupc_update_batch(self.h, e, o, n, None)
        ed = torch.from_numpy(e).cuda() if n else None
        od = torch.from_numpy(o).cuda() if n else None
        st = C.cupc_update_batch(self.h, ed, od, n, None)
        torch.cuda.synchronize()
        return st

    def query(self, pairs, host=False):
        p = np.ascontiguousarray(np.asarray(pairs, np.uint32).reshape(-1))
        m = p.size // 2
        if host:
            out = np.zeros(m, np.uint8)
            st = C.cupc_query(self.h, p, m, out, None)
            return st, out
        pd = torch.from_numpy(p).cuda()
        od = torch.zeros(m, dtype=torch.uint8, device="cuda")
        st = C.cupc_query(self.h, pd, m, od, None)
        torch.cuda.synchronize()
        return st, od.cpu().numpy()

    def forest(self):
        out = np.zeros(self.V, np.uint64)
        st, n = C.cupc_spanning_forest(self.h, out, self.V, None)
        return st, out[:n].copy()

    def labels(self):
        out = np.zeros(self.V, np.uint32)
        C.check(C.cupc_labels(self.h, out, None))
        return out

    def sync(self):
        return C.cupc_sync(self.h, None)

    def export(self):
        out = np.zeros((self.L, self.V, self.W, 2), np.uint64)
        C.check(C.cupc_export_sketches(self.h, out, out.nbytes, None))
        return out

    def stats(self):
        s = np.zeros(8, np.uint64)
        C.check(C.cupc_stats(self.h, s, None))
        return {"rounds": int(s[0]), "fail": int(s[1]), "false_pos": int(s[2]), "complete": bool(s[3]),
                "forest": int(s[4]), "recoveries": int(s[5]), "chunks": int(s[6]), "err": int(s[7])}

    def round_log(self):
        live = np.zeros(self.L, np.uint32)
        ncand = np.zeros(self.L, np.uint32)
        ids = np.zeros(self.L * self.V + 1, np.uint64)
        st, R = C.cupc_round_log(self.h, live, ncand, ids, ids.size, None)
        C.check(st)
        out, k = [], 0
        for r in range(R):
            n = int(ncand[r])
            out.append((int(live[r]), np.unique(ids[k:k + n])))
            k += n
        return out
