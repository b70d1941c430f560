"""GB300-native synchrotron ray march (synax, arXiv 2410.01136) -- placeholder."""
