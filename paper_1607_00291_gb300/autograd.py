"""torch.autograd.Function over tc_contract (filled in below)."""
import torch


class TcContract(torch.autograd.Function):
    pass


def contract_autograd(*a, **k):
    raise NotImplementedError
