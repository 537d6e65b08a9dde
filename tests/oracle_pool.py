"""The CPU oracle run on every host core, for parity tests at full workload
size (test infrastructure).

A job is a crop (y, x, h, w) of one image held in shared memory; a worker
runs ``oracle.label`` on the crop and returns the crop's counts and chip
counts and a digest of its labels (BLAKE2b, 128 bits), so that gigabytes
of labels need not travel between processes.  The GPU side digests its own
labels of the same crop; equal digests mean equal label maps.  A crop that
starts on the chip grid of the whole image (y, x multiples of the chip)
has the same chips as that region of the whole image, so a scene can be
checked as stripes of whole chip rows.

Workers are spawned, never forked: a CUDA context in the parent is not
inherited.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np


def digest(labels: np.ndarray) -> str:
    return hashlib.blake2b(np.ascontiguousarray(labels).tobytes(), digest_size=16).hexdigest()


def _job(task):
    name, shape, dtype, box, params = task
    from multiprocessing import shared_memory
    import oracle
    shm = shared_memory.SharedMemory(name=name)
    try:
        img = np.ndarray(shape, dtype=np.dtype(dtype), buffer=shm.buf)
        y, x, h, w = box
        crop = np.array(img[y:y + h, x:x + w], order="C", copy=True)  # not a view of shm
        del img
    finally:
        shm.close()
    lab, cnt, cc, _ = oracle.label(crop, params)
    return digest(lab), cnt, cc


def _ready(_):
    import oracle  # noqa: F401
    return os.getpid()


class OraclePool:
    def __init__(self, cores: int | None = None):
        import multiprocessing as mp
        self.cores = int(cores or len(os.sched_getaffinity(0)))
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_ready, range(self.cores), chunksize=1)

    def label_crops(self, img: np.ndarray, boxes, params=None):
        """oracle.label on every crop box of img; list of (digest, counts,
        chip_counts) in box order."""
        from multiprocessing import shared_memory
        shm = shared_memory.SharedMemory(create=True, size=img.nbytes)
        try:
            np.ndarray(img.shape, dtype=img.dtype, buffer=shm.buf)[...] = img
            tasks = [(shm.name, img.shape, img.dtype.str, tuple(int(v) for v in b), params)
                     for b in boxes]
            # largest crops first so the pool's last wave is short
            order = sorted(range(len(tasks)), key=lambda i: -boxes[i][2] * boxes[i][3])
            res = self.pool.map(_job, [tasks[i] for i in order], chunksize=1)
        finally:
            shm.close()
            shm.unlink()
        out = [None] * len(tasks)
        for i, r in zip(order, res):
            out[i] = r
        return out

    def label_stripes(self, img: np.ndarray, chip: int = 256, params=None):
        """The whole image as stripes of one chip row each: (per-stripe
        digests, counts[4], chip_counts[gy, gx, 4])."""
        H, W = img.shape[:2]
        boxes = [(y, 0, min(chip, H - y), W) for y in range(0, H, chip)]
        res = self.label_crops(img, boxes, params)
        cnt = np.zeros(4, np.uint64)
        for r in res:
            cnt += r[1]
        cc = np.concatenate([r[2] for r in res], axis=0)
        return [r[0] for r in res], cnt, cc

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
