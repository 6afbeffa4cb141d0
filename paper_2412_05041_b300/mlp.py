"""Learned ghost rejection: candidate collection, GPU training, threshold choice,
model files and evaluation.

The reconstruction's candidates (every track that passes the loose chi2/ndf
cut, before the 3-hit rule) are labelled by generator truth; a 12 -> 32 -> 32
-> 1 network is trained on the GPU by the library's own kernels
(``velo_mlp_loss_grad`` + ``velo_mlp_adam_step``, float32), and its logit
threshold is chosen so that the efficiency stays within a margin of the plain
chi2 method while the ghost rate drops.  Inference inside the reconstruction
runs on bfloat16 tensor cores (``velo_params_t.use_mlp``).
"""
from __future__ import annotations

import ctypes
import struct
from dataclasses import dataclass

import numpy as np
import torch

from . import MLP_FLOATS, MLP_WEIGHTS, N_FEATURES, check, default_params, lib
from .api import reconstruct
from . import truth

MAGIC = b"VELOMLP\0"
VERSION = 1


def _p(t: torch.Tensor) -> int:
    return int(t.data_ptr())


def _stream() -> int:
    return int(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------------ model files
def save(path: str, blob: np.ndarray, logit_min: float) -> None:
    """Binary model file: magic, version, n_floats, logit threshold, float32 blob."""
    blob = np.ascontiguousarray(blob, np.float32)
    assert blob.size == MLP_FLOATS
    with open(path, "wb") as f:
        f.write(MAGIC + struct.pack("<IIf", VERSION, blob.size, float(logit_min)) + blob.tobytes())


def load(path: str) -> tuple[np.ndarray, float]:
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError("not a ghost-rejection model file")
    version, n, thr = struct.unpack("<IIf", data[8:20])
    if version != VERSION or n != MLP_FLOATS:
        raise ValueError(f"model file version {version} / size {n} not supported")
    return np.frombuffer(data[20:20 + 4 * n], np.float32).copy(), thr


# ------------------------------------------------------------------ candidates
@dataclass
class Candidates:
    features: np.ndarray   # [N, 12] float32
    labels: np.ndarray     # [N] float32 (1 = matches a particle)
    batch: object          # generator batch (with truth)
    result: dict           # numpy result of the candidate reconstruction
    match: np.ndarray      # [N] matched batch-global particle id, -1 = ghost
    reconstructible: np.ndarray  # batch-global ids of reconstructible particles


def candidate_params(base=None):
    """The reconstruction's parameters for candidate collection: the 3-hit rule off."""
    p = base if base is not None else default_params()
    q = default_params(**{k: getattr(p, k) for k, _ in p._fields_})
    q.chi2ndf_max_3hit = q.chi2ndf_max
    q.use_mlp = 0
    return q


def collect(batch, params=None) -> Candidates:
    """Reconstruct `batch` (generator batch with truth) on the GPU without the
    3-hit rule and label every candidate by truth."""
    off = torch.from_numpy(batch.offsets.view(np.int64)).cuda()
    pix = torch.from_numpy(batch.pixels.view(np.int32)).cuda()
    r = reconstruct(off, pix, batch.geometry, candidate_params(params), pixel_labels=True, features=True)
    res = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items()}
    ct = truth.cluster_truth(batch, res)
    m = truth.track_matches(res, ct)
    rec = truth.reconstructible(batch, res, ct)
    return Candidates(res["track_features"].astype(np.float32), (m >= 0).astype(np.float32), batch, res, m, rec)


# ------------------------------------------------------------------ training
def init_weights(seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    w = np.zeros(MLP_WEIGHTS, np.float32)
    o = 0
    for fan_in, fan_out in ((N_FEATURES, 32), (32, 32)):
        n = fan_in * fan_out
        w[o:o + n] = rng.normal(0, np.sqrt(2.0 / fan_in), n)
        o += n + fan_out  # biases stay 0
    w[o:o + 32] = rng.normal(0, np.sqrt(1.0 / 32), 32)
    return w


def normalisation(features: np.ndarray):
    mean = features.astype(np.float64).mean(0)
    std = features.astype(np.float64).std(0)
    inv = np.where(std > 0, 1.0 / np.where(std > 0, std, 1.0), 1.0)
    return mean.astype(np.float32), inv.astype(np.float32)


class Trainer:
    """Adam on the library's loss/gradient kernels; all tensors on the current CUDA device."""

    def __init__(self, w0: np.ndarray, batch_size: int, lr: float = 3e-3, betas=(0.9, 0.999), eps: float = 1e-8):
        dev = torch.device("cuda")
        self.w = torch.from_numpy(np.asarray(w0, np.float32).copy()).to(dev)
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.g = torch.zeros_like(self.w)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        nbytes = ctypes.c_uint64()
        check(lib().velo_mlp_workspace_size(batch_size, ctypes.byref(nbytes)))
        self.ws = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
        self.batch_size, self.lr, self.betas, self.eps = batch_size, lr, betas, eps
        self.t = 0

    def loss_grad(self, x: torch.Tensor, y: torch.Tensor) -> None:
        check(lib().velo_mlp_loss_grad(_p(x), _p(y), x.shape[0], _p(self.w), _p(self.g), _p(self.loss), _p(self.ws),
                                       self.ws.numel(), _stream()), "velo_mlp_loss_grad")

    def step(self, x: torch.Tensor, y: torch.Tensor) -> None:
        self.loss_grad(x, y)
        self.t += 1
        check(lib().velo_mlp_adam_step(_p(self.w), _p(self.g), _p(self.m), _p(self.v), MLP_WEIGHTS, self.lr,
                                       self.betas[0], self.betas[1], self.eps, self.t, _stream()), "velo_mlp_adam_step")


def train(features: np.ndarray, labels: np.ndarray, epochs: int = 8, batch_size: int = 8192, lr: float = 3e-3,
          seed: int = 0) -> tuple[np.ndarray, list]:
    """Train on the GPU; returns (model blob, per-epoch mean loss)."""
    mean, inv = normalisation(features)
    dev = torch.device("cuda")
    X = (torch.from_numpy(features).to(dev) - torch.from_numpy(mean).to(dev)) * torch.from_numpy(inv).to(dev)
    Y = torch.from_numpy(labels.astype(np.float32)).to(dev)
    tr = Trainer(init_weights(seed), batch_size, lr)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    n = X.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen).to(dev)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch_size + 1, batch_size):
            idx = perm[b0:b0 + batch_size]
            tr.step(X[idx].contiguous(), Y[idx].contiguous())
            tot += float(tr.loss.item())
            cnt += 1
        hist.append(tot / max(cnt, 1))
    blob = np.concatenate([mean, inv, tr.w.cpu().numpy()]).astype(np.float32)
    return blob, hist


def infer(features: np.ndarray, blob: np.ndarray, mode: int = 0) -> np.ndarray:
    """Logits of raw features: mode 0 = bfloat16 tensor cores (as in the reconstruction), 1 = float32."""
    dev = torch.device("cuda")
    f = torch.from_numpy(np.ascontiguousarray(features, np.float32)).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(blob, np.float32)).to(dev)
    out = torch.empty(max(f.shape[0], 1), dtype=torch.float32, device=dev)
    check(lib().velo_mlp_infer(_p(f), f.shape[0], _p(b), _p(out), mode, _stream()), "velo_mlp_infer")
    return out[: f.shape[0]].cpu().numpy()


# ------------------------------------------------------------------ threshold and evaluation
def event_metrics_at(cands: Candidates, keep: np.ndarray) -> dict:
    """Efficiency / ghost rate of the candidate set restricted to `keep` (bool per candidate)."""
    mk = cands.match[keep]
    found = np.intersect1d(cands.reconstructible, mk[mk >= 0])
    return dict(efficiency=len(found) / max(len(cands.reconstructible), 1),
                ghost_rate=float((mk < 0).mean()) if len(mk) else 0.0, tracks=int(keep.sum()))


def plain_keep(cands: Candidates, cut3: float) -> np.ndarray:
    f = cands.features
    return ~((f[:, 0] == 3) & ~(f[:, 1] <= cut3))


def choose_threshold(cands: Candidates, logits: np.ndarray, cut3: float, margin: float = 0.0025) -> float:
    """Largest logit threshold whose efficiency is within `margin` of the plain method's."""
    eff_plain = event_metrics_at(cands, plain_keep(cands, cut3))["efficiency"]
    best = float(np.min(logits)) - 1.0
    for thr in np.quantile(logits, np.linspace(0.0, 0.3, 61)):
        if event_metrics_at(cands, logits >= thr)["efficiency"] >= eff_plain - margin:
            best = max(best, float(thr))
    return best
