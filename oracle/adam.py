"""Adam for the oracle (float64).  Test infrastructure only.

The paper solves every stage with an adaptive first-order method and cites
Adam (Sec. 1 and Sec. 3.2) without giving its constants; this is Adam as
Kingma & Ba define it, with bias correction:
    m <- b1 m + (1-b1) g ;  v <- b2 v + (1-b2) g^2
    x <- x - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
"""
import numpy as np


class Adam:
    def __init__(self, shape, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(shape)
        self.v = np.zeros(shape)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, x, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return x - self.lr * mh / (np.sqrt(vh) + self.eps)
