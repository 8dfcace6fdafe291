"""k-NN retrieval under the elastic distance with the learned pruning
network, against exact search (every gallery curve measured), and what the
network gains over pruning by the raw descriptors."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_17779_gb300 import knn, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def test_pruned_search_recall_and_gain():
    N, G, Q, band = 128, 1500, 40, 16
    gal = torch.from_numpy(synth.shape_gallery(1, G, N, device=DEV).curves).to(DEV)
    qry = torch.from_numpy(synth.shape_gallery(2, Q, N, device=DEV).curves).to(DEV)
    dg = knn.descriptors(gal)
    dq = knn.descriptors(qry, dg)
    exact, e_exact = knn.search(qry, gal, k=10, band=band)
    net, loss, n_train = knn.train_pruner(gal, dg, band=band, steps=1000, seed=3)
    rec = {}
    for n_cand in (60, 150):  # 4% and 10% of the gallery measured
        found, e_found = knn.search(qry, gal, k=10, band=band, n_cand=n_cand, qdesc=dq.x,
                                    gdesc=dg.x, net=net)
        raw, _ = knn.search(qry, gal, k=10, band=band, n_cand=n_cand, qdesc=dq.x, gdesc=dg.x)
        rec[n_cand] = (knn.recall_at_k(found, exact), knn.recall_at_k(raw, exact))
        print(f"recall@10 with {n_cand}/{G} candidates: network {rec[n_cand][0]:.4f}, raw "
              f"descriptors {rec[n_cand][1]:.4f}; training pairs {n_train}, loss {loss:.4f}")
    # the network's gain: the same recall from fewer elastic distances
    assert rec[60][0] >= rec[60][1] + 0.02
    assert rec[150][0] >= 0.99
    # the pruned search's distances are true elastic distances: spot-check
    # three queries' winners against the oracle
    for q in range(3):
        j = int(found[q, 0])
        o = oracle.elastic_pairs(qry[q].cpu().numpy(), gal[j].cpu().numpy(), band=band)
        assert abs(o["energy"][0] - e_found[q, 0].item()) < 1e-11
    # exact search returns its k best in ascending order
    assert (torch.diff(e_exact, dim=1) >= 0).all()
