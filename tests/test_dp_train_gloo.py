"""Data-parallel plumbing of the U-Net training step on CPU, two gloo ranks
(Sec. III-C "Distributed U-Net Model Training using Horovod Framework":
rank 0's initial weights go to every worker, each worker computes the
gradient of its own batch, the gradients are averaged, every worker applies
the same update).  The oracle's backward pass on a tiny network stands in
for the GPU step; the package's averaging, broadcast and step functions are
the ones the GPU trainer runs."""
import os
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _OracleTrainer:
    """The Trainer interface (params / set_params / backward / adam) over the
    oracle, on a 16 x 16 input with a depth-2, width-4 network."""

    def __init__(self, seed):
        import synth
        self.wts = synth.unet_weights(4, 2, seed=seed)
        self.names = list(self.wts)
        self.t = 0
        self.m = self.v = None
        self.seen = []

    def _flat(self, d):
        return torch.tensor(np.concatenate([np.concatenate([np.ravel(w), np.ravel(b)])
                                            for w, b in (d[k] for k in self.names)]))

    def _unflat(self, flat):
        a = flat.numpy().astype(np.float64)
        out, o = {}, 0
        for k in self.names:
            w, b = self.wts[k]
            nw, nb = w.size, b.size
            out[k] = (a[o:o + nw].reshape(w.shape), a[o + nw:o + nw + nb])
            o += nw + nb
        return out

    def params(self):
        return self._flat(self.wts).double()

    def set_params(self, flat):
        self.wts = self._unflat(flat)
        self.t = 0
        self.m = self.v = None

    def backward(self, chips, labels, grads=None, loss=None, stream=None):
        import oracle.unet_train as T
        acts, logits = T.forward_saved(chips, self.wts, 2)
        lo, g = T.backward_network(acts, logits, labels, self.wts, 2)
        return self._flat(g).double(), torch.tensor([lo])

    def adam(self, grads, lr=1e-3, t=None, stream=None):
        import oracle.unet_train as T
        self.seen.append(grads.clone())
        self.t += 1
        p = self.params().numpy()
        g = grads.numpy()
        m = np.zeros_like(p) if self.m is None else self.m
        v = np.zeros_like(p) if self.v is None else self.v
        p, self.m, self.v = T.adam_step(p, g, m, v, self.t, lr)
        self.wts = self._unflat(torch.tensor(p))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle.unet_train as T
    import paper_2403_13135_gb300 as sil

    # averaging: the mean of the ranks' tensors on every rank
    g = torch.arange(6, dtype=torch.float32) * (rank + 1)
    sil.average_gradients_(g)
    ok_avg = torch.allclose(g, torch.arange(6, dtype=torch.float32) * 1.5)

    # broadcast: every rank starts from rank 0's weights (seeds differ)
    tr = _OracleTrainer(seed=100 + rank)
    p0 = sil.broadcast_params_(tr)

    # two data-parallel steps, each rank on its own batch
    rng = np.random.default_rng(7 + rank)
    losses = []
    grads_seen = []
    for _ in range(2):
        x = rng.random((1, 16, 16, 3))
        lab = rng.integers(0, 4, (1, 16, 16))
        # the mean over ranks the oracle computes, for comparison
        _, glocal = T.backward_network(*T.forward_saved(x, tr.wts, 2), lab, tr.wts, 2)
        flat_local = tr._flat(glocal).double()
        both = [torch.zeros_like(flat_local) for _ in range(world)]
        dist.all_gather(both, flat_local)
        losses.append(float(sil.Trainer.step(tr, x, lab, lr=1e-3).item()))
        grads_seen.append((tr.seen[-1], sum(both) / world))
    ok_mean = all(torch.allclose(a, b, rtol=1e-12, atol=0) for a, b in grads_seen)
    q.put((rank, ok_avg, p0.numpy(), tr.params().numpy(), ok_mean, losses))
    dist.destroy_process_group()


def test_two_rank_data_parallel_steps():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 28500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a0, p00, p10, m0, l0), (_, a1, p01, p11, m1, l1) = res
    assert a0 and a1                         # all-reduce mean
    assert np.array_equal(p00, p01)          # rank 0's initial weights everywhere
    assert m0 and m1                         # Adam saw the mean of both ranks' gradients
    assert np.array_equal(p10, p11)          # same update on every rank
    assert l0 != l1                          # each rank's loss is its own batch's
