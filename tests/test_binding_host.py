"""Host-side pieces of the Python binding that need no GPU."""
import torch

from paper_2603_00477_gb300 import binding as B


def test_resolve_device_fills_the_cuda_index(monkeypatch):
    """"cuda" names the current device, so a plan's workspace on cuda:N is
    kept (not re-allocated) when a later call names "cuda" again."""
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)
    assert B._resolve_device("cuda") == torch.device("cuda", 3)
    assert B._resolve_device(torch.device("cuda")) == torch.device("cuda", 3)
    assert B._resolve_device("cuda:1") == torch.device("cuda", 1)
    assert B._resolve_device("cpu") == torch.device("cpu")
    assert torch.device("cuda") != torch.device("cuda", 3)  # why the index must be filled in


class _FakeTensor:
    def __init__(self, n, device):
        self.n, self.device = n, torch.device(device)

    def numel(self):
        return self.n

    def data_ptr(self):
        return 4096


def _fake_batch(monkeypatch, calls):
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch, "empty", lambda n, dtype=None, device=None: _FakeTensor(n, device))
    monkeypatch.setattr(B, "stencil_batch_workspace_bytes", lambda h, steps: 100)
    monkeypatch.setattr(B, "stencil_batch_set_workspace", lambda h, p, n: calls.append((p, n)))
    batch = object.__new__(B.Batch)
    batch.handle = None
    batch._ws = None
    return batch


def test_batch_workspace_follows_the_device(monkeypatch):
    """A batch's workspace is re-allocated when the inputs move to another
    device, and kept when "cuda" names the device it is already on."""
    calls = []
    batch = _fake_batch(monkeypatch, calls)
    ws0 = batch.ensure_workspace(3, "cuda:0")
    assert ws0.device == torch.device("cuda", 0) and len(calls) == 1
    assert batch.ensure_workspace(3, "cuda") is ws0 and len(calls) == 1
    ws1 = batch.ensure_workspace(3, torch.device("cuda", 1))
    assert ws1 is not ws0 and ws1.device == torch.device("cuda", 1) and len(calls) == 2
