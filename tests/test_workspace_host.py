"""Workspace queries are host arithmetic (no device work): the phased batch
and the host-buffer call size what they hold across their steps."""
import torch

import paper_1612_08709_gb300 as pkg


def test_phased_batch_workspace_holds_member_state():
    shapes = [(20000, 100), (5000, 256), (3000, 16)]
    ws = pkg.ts_svd_batched_workspace_size(shapes, mode="fp64_tc")
    # per member: B, the factor X, J, V~, W (n x n doubles) and, from
    # n = 64, the FP32 phase's 2 n^2 floats and 2 n^2 doubles
    state = sum(5 * n * n * 8 + (3 * n * n * 8 if n >= 64 else 0) for _, n in shapes)
    assert ws >= state
    # FP32 storage keeps Y~ (m x n doubles) in the workspace as well
    ws32 = pkg.ts_svd_batched_workspace_size(shapes, dtype=torch.float32, mode="fp64_tc")
    assert ws32 >= ws + sum(m * n * 8 for m, n in shapes) - 256 * len(shapes)


def test_host_call_workspace_holds_device_copies():
    m, n = 100000, 200
    ws = pkg.ts_svd_host_workspace_size(m, n)
    assert ws >= 2 * m * n * 8 + pkg.ts_svd_workspace_size(m, n) - 256
