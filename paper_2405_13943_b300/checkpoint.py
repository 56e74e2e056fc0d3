"""Checkpoint and resume of a batched DOGS run.

A checkpoint holds everything the next iteration reads: the global model z,
the block-local copies x_k, the scaled duals u_k, Adam's moments m and v,
the iteration counter t and the penalties rho (with the adaptive-penalty
state of Eq. 10 when it is on), and with densification the statistics
accumulated since the last one.  After a densification changed the block
layout, the layout itself (the sharing map) is stored too: a trainer built
on the run's original layout takes it on load.  The anchors z - u are not stored: after a
load they are rebuilt by dg_admm_anchor, the same single subtraction the
consensus writes, so they come back bit for bit.  Gradients are scratch and
are not stored either.

File layout (little endian):
    8 bytes   magic "DOGSCKPT"
    8 bytes   uint64 length H of the header
    8 bytes   uint64 start of the data area (a multiple of 4096)
    H bytes   UTF-8 JSON header: format version, t, rho, the run's
              configuration, fingerprints of the block split and of the
              run's original split, and for each buffer and array its name,
              byte offset in the data area, byte length, dtype and shape
              (arrays) and CRC-32
    ...       raw buffers, each starting on a 4096-byte boundary, in the
              library's device layout (padding lanes included)
The file is written to `path + ".tmp"` and renamed into place, so a crash
mid-write leaves the previous checkpoint intact.  Loading checks the
magic, the version, the split fingerprint, the configuration, every
buffer's size and CRC before anything on the device is overwritten.
"""
from __future__ import annotations

import json
import os
import struct
import zlib
from typing import Dict, List

import numpy as np
import torch

from . import dogs as D
from . import synth as S

MAGIC = b"DOGSCKPT"
VERSION = 2
READABLE = (1, 2)
ALIGN = 4096
CHUNK = 64 << 20          # bytes staged through host memory at a time
BUFFERS = ("z", "x", "u", "m", "v")
CONFIG = ("lr", "alpha", "intv", "loss_kind", "w_l1", "w_ssim", "bg")


class CheckpointError(RuntimeError):
    pass


def split_fingerprint(split) -> str:
    crc = 0
    for a in (split.copy_gid, split.blk_off, split.blk_nshared, split.g_off, split.g_copies):
        crc = zlib.crc32(np.ascontiguousarray(a).tobytes(), crc)
    return f"{crc:08x}:{split.K}:{split.n_copies}:{int(split.n_shared_globals)}"


def _config(tr) -> Dict:
    return {k: (list(getattr(tr, k)) if isinstance(getattr(tr, k), (list, tuple)) else getattr(tr, k))
            for k in CONFIG}


def _chunks(t: torch.Tensor):
    flat = t.reshape(-1).view(torch.uint8)
    for b in range(0, flat.numel(), CHUNK):
        yield flat[b:b + CHUNK]


SPLIT_ARRAYS = ("copy_gid", "blk_off", "blk_nshared", "g_off", "g_copies", "cells")


def _arrays(tr) -> Dict[str, np.ndarray]:
    """Host arrays stored beside the buffers: the block layout when it is not
    the run's original one, and the densification statistics."""
    out: Dict[str, np.ndarray] = {}
    origin = getattr(tr, "split_origin", None)
    if origin is not None and origin != split_fingerprint(tr.split):
        for name in SPLIT_ARRAYS:
            out["split." + name] = np.ascontiguousarray(getattr(tr.split, name))
    if getattr(tr, "dstats", None) is not None:
        out["dstats"] = tr.dstats.detach().cpu().numpy()
    return out


def save(tr, path: str) -> None:
    """Write the state of DogsTrainer `tr` after its last completed iteration
    (one pass over the device data: the CRCs are fixed-width hex, so the
    header is written with placeholders and rewritten in place at the end)."""
    bufs = {name: getattr(tr, name) for name in BUFFERS}
    on_gpu = bufs["z"].data.is_cuda
    if on_gpu:
        torch.cuda.synchronize()
    if hasattr(tr, "current_rho"):
        tr.current_rho()                 # rho as Eq. 10 left it on the device
    entries: List[Dict] = []
    off = 0
    for name, b in bufs.items():
        nbytes = b.data.numel() * 4
        entries.append(dict(name=name, n=b.n, ld=b.ld, deg=b.deg, nbytes=nbytes, offset=off, crc32="0" * 8))
        off += -(-nbytes // ALIGN) * ALIGN          # offsets relative to the data start
    arrays = _arrays(tr)
    arr_entries: List[Dict] = []
    for name, a in arrays.items():
        arr_entries.append(dict(name=name, dtype=str(a.dtype), shape=list(a.shape), nbytes=int(a.nbytes),
                                offset=off, crc32="0" * 8))
        off += -(-int(a.nbytes) // ALIGN) * ALIGN
    ad = tr.adaptive
    header = dict(format="dogs-checkpoint", version=VERSION, t=int(tr.t), rho=[float(r) for r in tr.rho],
                  adaptive=None if ad is None else dict(rho=list(ad.rho), mu=ad.mu, tau_inc=ad.tau_inc,
                                                        tau_dec=ad.tau_dec, freeze_after=ad.freeze_after),
                  config=_config(tr), split=split_fingerprint(tr.split),
                  split_origin=getattr(tr, "split_origin", None),
                  split_scalars=dict(n_shared_globals=int(tr.split.n_shared_globals), band=float(tr.split.band)),
                  buffers=entries, arrays=arr_entries)
    hdr = json.dumps(header, sort_keys=True).encode()
    data_start = -(-(24 + len(hdr)) // ALIGN) * ALIGN
    staging = torch.empty(CHUNK, dtype=torch.uint8, pin_memory=on_gpu)
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(MAGIC + struct.pack("<QQ", len(hdr), data_start) + hdr)
        for e in entries:
            f.seek(data_start + e["offset"])
            crc = 0
            for c in _chunks(bufs[e["name"]].data):
                h = staging[:c.numel()]
                h.copy_(c)
                crc = zlib.crc32(h.numpy(), crc)
                f.write(h.numpy().tobytes())
            e["crc32"] = f"{crc:08x}"
        for e in arr_entries:
            raw = np.ascontiguousarray(arrays[e["name"]]).tobytes()
            f.seek(data_start + e["offset"])
            f.write(raw)
            e["crc32"] = f"{zlib.crc32(raw):08x}"
        last = (arr_entries or entries)[-1]
        f.truncate(data_start + last["offset"] + last["nbytes"])
        final = json.dumps(header, sort_keys=True).encode()
        assert len(final) == len(hdr)
        f.seek(24)
        f.write(final)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def read_header(path: str) -> Dict:
    with open(path, "rb") as f:
        head = f.read(24)
        if len(head) < 24 or head[:8] != MAGIC:
            raise CheckpointError(f"{path}: not a DOGS checkpoint")
        hlen, data_start = struct.unpack("<QQ", head[8:])
        raw = f.read(hlen)
    if len(raw) != hlen:
        raise CheckpointError(f"{path}: truncated header")
    header = json.loads(raw.decode())
    header["data_start"] = data_start
    if header.get("format") != "dogs-checkpoint" or header.get("version") not in READABLE:
        raise CheckpointError(f"{path}: unsupported format {header.get('format')} v{header.get('version')}")
    return header


def load(tr, path: str) -> Dict:
    """Restore DogsTrainer `tr` (built on the same split, views and targets)
    from `path`.  Everything is verified on the host before the device
    buffers are written.  Returns the header."""
    header = read_header(path)
    size = os.path.getsize(path)
    arrays: Dict[str, np.ndarray] = {}
    with open(path, "rb") as f:
        for e in header.get("arrays", []):
            at = header["data_start"] + e["offset"]
            if at + e["nbytes"] > size:
                raise CheckpointError(f"array {e['name']}: file truncated")
            f.seek(at)
            raw = f.read(e["nbytes"])
            if f"{zlib.crc32(raw):08x}" != e["crc32"]:
                raise CheckpointError(f"array {e['name']}: CRC mismatch")
            arrays[e["name"]] = np.frombuffer(raw, np.dtype(e["dtype"])).reshape(e["shape"]).copy()
    new_split = None
    if header["split"] != split_fingerprint(tr.split):
        # a densified layout of the same run: taken when the trainer was built on the run's original layout
        if (header.get("split_origin") is None or header.get("split_origin") != getattr(tr, "split_origin", None)
                or "split.copy_gid" not in arrays):
            raise CheckpointError("checkpoint was written for another block split")
        sc = header["split_scalars"]
        new_split = S.BlockSplit(*(arrays["split." + n] for n in SPLIT_ARRAYS[:5]), int(sc["n_shared_globals"]),
                                 arrays["split.cells"], float(sc["band"]))
        if split_fingerprint(new_split) != header["split"]:
            raise CheckpointError("stored block split does not match its fingerprint")
    cfg, want = header["config"], _config(tr)
    diff = [k for k in CONFIG if json.loads(json.dumps(want[k])) != cfg[k]]
    if diff:
        raise CheckpointError(f"configuration differs from the checkpoint's: {diff}")
    if (header["adaptive"] is None) != (tr.adaptive is None):
        raise CheckpointError("adaptive penalty on in one of checkpoint and trainer only")
    if ("dstats" in arrays) != (getattr(tr, "dstats", None) is not None):
        raise CheckpointError("densification on in one of checkpoint and trainer only")
    # the shape each buffer must have: the trainer's own, or for a stored
    # layout the one that layout implies (globals for z, copies for the rest)
    if new_split is None:
        want_shape = {n: (getattr(tr, n).n, getattr(tr, n).ld, getattr(tr, n).deg, getattr(tr, n).data.numel() * 4)
                      for n in BUFFERS}
        n_copies = tr.split.n_copies
    else:
        deg = tr.z.deg
        n_glob = len(new_split.g_off) - 1
        n_copies = new_split.n_copies
        want_shape = {}
        for e in header["buffers"]:
            n = n_glob if e["name"] == "z" else n_copies
            ld = int(e["ld"])
            if ld < n or ld % 4:
                raise CheckpointError(f"buffer {e['name']}: leading dimension {ld} does not fit {n}")
            want_shape[e["name"]] = (n, ld, deg, ld * (12 + 3 * (deg + 1) ** 2) * 4)
    if sorted(e["name"] for e in header["buffers"]) != sorted(BUFFERS):
        raise CheckpointError("checkpoint does not hold every parameter buffer")
    if "dstats" in arrays and arrays["dstats"].size != 2 * max(n_copies, 1):
        raise CheckpointError("densification statistics: size differs from the layout's")
    # every buffer read and verified on the host before anything of the trainer changes
    host: Dict[str, np.ndarray] = {}
    with open(path, "rb") as f:
        for e in header["buffers"]:
            if (e["n"], e["ld"], e["deg"], e["nbytes"]) != want_shape[e["name"]]:
                raise CheckpointError(f"buffer {e['name']}: shape differs from the trainer's")
            at = header["data_start"] + e["offset"]
            if at + e["nbytes"] > size:
                raise CheckpointError(f"buffer {e['name']}: file truncated")
            f.seek(at)
            raw = f.read(e["nbytes"])
            if f"{zlib.crc32(raw):08x}" != e["crc32"]:
                raise CheckpointError(f"buffer {e['name']}: CRC mismatch")
            host[e["name"]] = np.frombuffer(raw, np.float32)
    if new_split is not None:
        dev = tr.z.data.device
        fresh = {e["name"]: D.GaussianBuffer(e["n"], e["deg"], dev, e["ld"]) for e in header["buffers"]}
        tr.install_split(new_split, fresh["z"], fresh["x"], fresh["m"], fresh["v"], fresh["u"], calibrate=False)
    for name, a in host.items():
        getattr(tr, name).data.copy_(torch.from_numpy(a.copy()))
    if "dstats" in arrays and getattr(tr, "dstats", None) is not None:
        tr.dstats.copy_(torch.from_numpy(arrays["dstats"]))
    tr.t = int(header["t"])
    tr.rho = [float(r) for r in header["rho"]]
    if tr.adaptive is not None:
        ad = header["adaptive"]
        tr.adaptive.rho = list(ad["rho"])
        tr.adaptive.mu, tr.adaptive.tau_inc, tr.adaptive.tau_dec = ad["mu"], ad["tau_inc"], ad["tau_dec"]
        tr.adaptive.freeze_after = ad["freeze_after"]
    tr.refresh_anchor()
    tr.graphs.clear()
    if new_split is not None and hasattr(tr, "calibrate_capacity"):
        tr.calibrate_capacity()                    # the instance capacity of the loaded state
    return header
