"""Batched contractions (filled in below)."""


class Plan:
    pass


def contract_batched(*a, **k):
    raise NotImplementedError
