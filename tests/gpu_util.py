"""Buffers for GPU tests: torch provides device and page-locked memory (plumbing only);
payloads come from the seeded generator, expectations from the oracle."""
import numpy as np
import torch

import payload

GUARD = 4096
CANARY = 0xA5


class Buf:
    """A byte buffer with canary guard bytes on both sides."""

    def __init__(self, n: int, where: str, offset: int = 0):
        self.n, self.where, self.offset = n, where, offset
        total = n + 2 * GUARD + 64
        if where == "dev":
            self.t = torch.full((total,), CANARY, dtype=torch.uint8, device="cuda")
        elif where == "pageable":  # ordinary host memory, not page-locked
            self.t = torch.full((total,), CANARY, dtype=torch.uint8)
        else:
            self.t = torch.full((total,), CANARY, dtype=torch.uint8).pin_memory()
        self.start = GUARD + offset
        self.view = self.t[self.start:self.start + n]

    @property
    def ptr(self) -> int:
        return self.t.data_ptr() + self.start

    def fill(self, data: np.ndarray) -> None:
        src = torch.from_numpy(np.ascontiguousarray(data).view(np.uint8))
        self.view.copy_(src)
        torch.cuda.synchronize()

    def numpy(self) -> np.ndarray:
        torch.cuda.synchronize()
        return self.t.cpu().numpy()[self.start:self.start + self.n] if self.where == "dev" \
            else self.t.numpy()[self.start:self.start + self.n].copy()

    def guards_intact(self) -> bool:
        torch.cuda.synchronize()
        a = self.t.cpu().numpy() if self.where == "dev" else self.t.numpy()
        return bool((a[:self.start] == CANARY).all() and (a[self.start + self.n:] == CANARY).all())


def seeded(kind: str, seed: int, n: int) -> np.ndarray:
    return payload.fill(kind, seed, n)
