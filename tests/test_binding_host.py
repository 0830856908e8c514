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
