"""GB300-native (sm_103a) particle -> IFU data-cube forward model (arXiv 2412.08265)."""
