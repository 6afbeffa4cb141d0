"""Train the ghost-rejection network on the GPU and write the model file.

    python -m paper_2412_05041_b300.train_ghost_mlp [--train-events 4200] [--test-events 1050]
           [--out paper_2412_05041_b300/models/ghost_mlp.bin] [--report report.json]

Candidates come from pile-up-5.5 events (the 10k-event benchmark workload's
generator settings): seed 4 for training (about 1M candidates), seed 5 for
testing (a fifth of that).  The network is trained by the library's own
kernels; its logit threshold is the largest that keeps the training-set
efficiency within 0.25 % of the plain chi2 method.  The report gives the loss
history and, on the test events, efficiency and ghost rate of the plain
method and of the learned one.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import velogen  # noqa: E402

from paper_2412_05041_b300 import build, mlp  # noqa: E402

DEFAULT_MODEL = os.path.join(HERE, "models", "ghost_mlp.bin")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-events", type=int, default=4200)
    ap.add_argument("--test-events", type=int, default=1050)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--report", default=None)
    a = ap.parse_args(argv)
    build()
    t0 = time.time()
    tr = mlp.collect(velogen.generate(velogen.Config(seed=4, n_events=a.train_events), truth=True))
    te = mlp.collect(velogen.generate(velogen.Config(seed=5, n_events=a.test_events), truth=True))
    t1 = time.time()
    blob, hist = mlp.train(tr.features, tr.labels, epochs=a.epochs, batch_size=a.batch, lr=a.lr)
    t2 = time.time()
    thr = mlp.choose_threshold(tr, mlp.infer(tr.features, blob, 0), cut3=2.0)
    z = mlp.infer(te.features, blob, 0)
    plain = mlp.event_metrics_at(te, mlp.plain_keep(te, 2.0))
    learned = mlp.event_metrics_at(te, z >= thr)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    mlp.save(a.out, blob, thr)
    rep = dict(train_candidates=int(len(tr.labels)), train_ghost_fraction=float(1 - tr.labels.mean()),
               test_candidates=int(len(te.labels)), epochs=a.epochs, batch=a.batch, lr=a.lr, loss_history=hist,
               logit_min=thr, test_plain=plain, test_learned=learned, collect_s=t1 - t0, train_s=t2 - t1)
    print(json.dumps(rep))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
