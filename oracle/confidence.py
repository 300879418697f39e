"""Oracle confidence-weighted objective (Eq. 5), for the training loop's next kernel.

TEST INFRASTRUCTURE (see the package docstring).  Plain PyTorch CPU ops in float64; autograd
on them supplies the gradient.

Sec. 4.2 (confidence-weighted optimisation): a network g: R^3 -> R with one hidden layer of
32 units maps a sample's position to C = 1 + exp(g) > 1, and the objective is
C L_task - alpha log C with alpha = 0.3.  Readings:
  - the position is the query position of the sample (the transmitter in these workloads,
    the receiver in the paper's moving-receiver setting), hidden activation ReLU (unstated);
  - over a batch of samples the objective is the mean of the per-sample objectives;
  - the reported confidence is min-max normalised over an evaluation set,
    (C - C_min) / (C_max - C_min).
"""
from __future__ import annotations

import torch

ALPHA = 0.3


def network(pos, W1, b1, W2, b2):
    """g(pos) = W2^T relu(W1^T pos + b1) + b2 for positions [B, 3] -> [B] (W input-major)."""
    return (torch.relu(pos @ W1 + b1) @ W2 + b2).reshape(-1)


def confidence(pos, weights):
    return 1.0 + torch.exp(network(pos, *weights))


def objective(pos, weights, task_loss, alpha=ALPHA):
    """Mean over samples of C L_task - alpha log C; task_loss [B]."""
    C = confidence(pos, weights)
    return (C * task_loss - alpha * torch.log(C)).mean()


def normalised(C):
    """(C - C_min) / (C_max - C_min) over the given set."""
    return (C - C.min()) / (C.max() - C.min())
